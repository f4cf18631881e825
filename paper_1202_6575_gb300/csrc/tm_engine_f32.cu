// Persistent tile-engine kernels for float keys.
#include "tm_engine_launch.cuh"

namespace pmerge {
template tm_status launch_engine<float>(const EngineArgs&, const tm_config*, cudaStream_t);
template tm_status launch_engine_fused<float>(const EngineArgs&, cudaStream_t);
}  // namespace pmerge
