// The resident schedule for FP32 messages (see mbp_resident.cuh).
#include "mbp_resident.cuh"

namespace mbp {

size_t resident_ctl_bytes() { return sizeof(ResidentCtl); }

int resident_error(const void* ctl_host) { return static_cast<const ResidentCtl*>(ctl_host)->error; }

template int resident_group<float>(const DevCode&, int);
template cudaError_t launch_resident_any<float>(const DevCode&, const DevState&, const DecodeArgs&, int, double,
                                                cudaStream_t);

}  // namespace mbp
