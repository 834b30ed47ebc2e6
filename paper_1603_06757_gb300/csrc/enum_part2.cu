// enum_part2.cu -- instantiations of the level enumerator for 9..12 32-bit words per row
// (split over several translation units so the build compiles them in parallel).
#include "enum_kernel.cuh"

namespace mdist {
template cudaError_t launch_nw<9>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<10>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<11>(const EnumParams &, int, bool, int, int, cudaStream_t);
template cudaError_t launch_nw<12>(const EnumParams &, int, bool, int, int, cudaStream_t);
}  // namespace mdist
