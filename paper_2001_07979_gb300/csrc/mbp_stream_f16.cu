// Streaming schedule with __half message storage and float arithmetic (see mbp_stream.cuh).
#include "mbp_stream.cuh"

namespace mbp {

template <>
int stream_iterations<float, __half>(const DevCode& c, DevState& st, const DecodeArgs& a, bool fixed, double l_max,
                                 float qscale, float inv_qscale, cudaStream_t s) {
  return stream::run<float, __half>(c, st, a, fixed, l_max, qscale, inv_qscale, s);
}

template <>
cudaError_t stream_group_step<float, __half>(const DevCode& c, const DevState& st, int first_iter, double l_max,
                                         cudaStream_t s, const StreamFork* fork) {
  return stream::group_step<float, __half>(c, st, first_iter, l_max, s, fork);
}

}  // namespace mbp
