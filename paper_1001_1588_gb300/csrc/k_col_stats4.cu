// Instantiation of the column stats pass for up to 4 observed block(s).
#include "k_cols.cuh"

namespace fftenkf {
cudaError_t col_stats_nobs4(const ColStatsParams& p, cudaStream_t s) { return col_stats_dispatch<4>(p, s); }
}  // namespace fftenkf
