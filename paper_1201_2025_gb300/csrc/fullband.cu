// Full-band detectors (dim > 8): placeholder until the CTA-per-pixel path lands.
#include "internal.h"

namespace wdad {
size_t fullband_workspace_bytes(const FullArgs&, int) { return 0; }
cudaError_t launch_detect_full(const FullArgs&, void*, size_t, int, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace wdad
