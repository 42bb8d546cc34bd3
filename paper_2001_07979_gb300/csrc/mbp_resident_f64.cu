// The resident schedule for FP64 messages (see mbp_resident.cuh).
#include "mbp_resident.cuh"

namespace mbp {

template int resident_group<double>(const DevCode&, int);
template cudaError_t launch_resident_any<double>(const DevCode&, const DevState&, const DecodeArgs&, int, double,
                                                 cudaStream_t);

}  // namespace mbp
