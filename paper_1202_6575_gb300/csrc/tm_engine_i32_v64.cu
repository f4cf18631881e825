// Persistent tile-engine kernels for int32_t keys with 8-byte payloads.
#include "tm_engine_launch.cuh"

namespace pmerge {
template tm_status launch_engine_v64<int32_t>(const EngineArgs&, const tm_config*, cudaStream_t);
template tm_status launch_engine_fused_v64<int32_t>(const EngineArgs&, cudaStream_t);
}  // namespace pmerge
