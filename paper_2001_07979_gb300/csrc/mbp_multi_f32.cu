// Grouped-decode kernels for float message storage (see mbp_multi.cuh).
#include "mbp_multi.cuh"

namespace mbp {
template struct MultiLaunch<float>;
}  // namespace mbp
