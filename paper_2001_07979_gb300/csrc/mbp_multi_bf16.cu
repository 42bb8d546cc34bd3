// Grouped-decode kernels for __nv_bfloat16 message storage (see mbp_multi.cuh).
#include "mbp_multi.cuh"

namespace mbp {
template struct MultiLaunch<__nv_bfloat16>;
}  // namespace mbp
