// enum_part1.cu -- instantiations of the level enumerator for 5..8 32-bit words per row
// (split over several translation units so the build compiles them in parallel).
#include "enum_kernel.cuh"

namespace mdist {
template cudaError_t launch_nw<5>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<6>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<7>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<8>(const EnumParams &, int, bool, int, int, cudaStream_t);
}  // namespace mdist
