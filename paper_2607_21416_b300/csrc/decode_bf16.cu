// decode_bf16.cu -- BF16 tensor-core anchor decoding (FP32 accumulation).
#include "gs_internal.cuh"

namespace gs {

int launch_decode_bf16(const DecodeArgs &a, cudaStream_t s)
{
    (void)a; (void)s;
    return GS_ERR_UNSUPPORTED;
}

}  // namespace gs
