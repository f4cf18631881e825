// Persistent tile-engine kernels for int32_t keys.
#include "tm_engine_launch.cuh"

namespace pmerge {
template tm_status launch_engine<int32_t>(const EngineArgs&, const tm_config*, cudaStream_t);
template tm_status launch_engine_fused<int32_t>(const EngineArgs&, cudaStream_t);
}  // namespace pmerge
