// Persistent tile-engine kernels for float keys with 8-byte payloads.
#include "tm_engine_launch.cuh"

namespace pmerge {
template tm_status launch_engine_v64<float>(const EngineArgs&, const tm_config*, cudaStream_t);
template tm_status launch_engine_fused_v64<float>(const EngineArgs&, cudaStream_t);
}  // namespace pmerge
