// Four-run tile-engine kernels (fused merge-sort rounds) for uint64_t keys.
#include "tm_engine4_launch.cuh"

namespace pmerge {
template tm_status launch_engine4<uint64_t>(const Engine4Args&, int, const tm_config*, cudaStream_t);
}  // namespace pmerge
