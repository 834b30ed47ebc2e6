// enum_part0.cu -- instantiations of the level enumerator for 1..4 32-bit words per row
// (split over several translation units so the build compiles them in parallel).
#include "enum_kernel.cuh"

namespace mdist {
template cudaError_t launch_nw<1>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<2>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<3>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<4>(const EnumParams &, int, bool, int, int, cudaStream_t);
}  // namespace mdist
