// Instantiation of the column stats pass for up to 2 observed block(s).
#include "k_cols.cuh"

namespace fftenkf {
cudaError_t col_stats_nobs2(const ColStatsParams& p, cudaStream_t s) { return col_stats_dispatch<2>(p, s); }
}  // namespace fftenkf
