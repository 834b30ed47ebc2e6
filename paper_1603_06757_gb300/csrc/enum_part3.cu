// enum_part3.cu -- instantiations of the level enumerator for 13..16 32-bit words per row
// (split over several translation units so the build compiles them in parallel).
#include "enum_kernel.cuh"

namespace mdist {
template cudaError_t launch_nw<13>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<14>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<15>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<16>(const EnumParams &, int, bool, int, int, cudaStream_t);
}  // namespace mdist
