// Instantiation of the column stats pass for up to 1 observed block(s).
#include "k_cols.cuh"

namespace fftenkf {
cudaError_t col_stats_nobs1(const ColStatsParams& p, cudaStream_t s) { return col_stats_dispatch<1>(p, s); }
}  // namespace fftenkf
