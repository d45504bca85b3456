// Tensor-map encoding for the TMA loads of the tensor-core kernels:
// cuTensorMapEncodeTiled, looked up from the driver through the runtime.
#pragma once

#include <cuda.h>

namespace hyde {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// nullptr when the driver does not provide it
EncodeTiledFn encode_tiled_fn();

}  // namespace hyde
