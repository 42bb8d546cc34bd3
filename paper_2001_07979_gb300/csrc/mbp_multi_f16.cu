// Grouped-decode kernels for __half message storage (see mbp_multi.cuh).
#include "mbp_multi.cuh"

namespace mbp {
template struct MultiLaunch<__half>;
}  // namespace mbp
