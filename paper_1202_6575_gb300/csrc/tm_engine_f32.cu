// Persistent tile-engine kernels for float keys with 4-byte payloads (and
// keys-only merges).
#include "tm_engine_launch.cuh"

namespace pmerge {
extern template tm_status launch_engine_v64<float>(const EngineArgs&, const tm_config*, cudaStream_t);
extern template tm_status launch_engine_fused_v64<float>(const EngineArgs&, cudaStream_t);
template tm_status launch_engine<float>(const EngineArgs&, const tm_config*, cudaStream_t);
template tm_status launch_engine_fused<float>(const EngineArgs&, cudaStream_t);
}  // namespace pmerge
