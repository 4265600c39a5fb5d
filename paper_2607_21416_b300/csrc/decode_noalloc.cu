// decode_noalloc.cu -- gs_decode_noalloc: the decode entry point for callers
// that cannot allocate device memory.
//
// Some hosts of this library cannot call cudaMalloc (or any allocator) at the
// moment they decode: a real-time mapping thread that must never block in the
// driver's allocator, a plug-in running inside a framework whose device memory
// is fully reserved by that framework's own pool, or code that must keep its
// device footprint fixed after start-up.  This entry point needs no workspace
// argument: its scratch (the per-view, per-2048-anchor visibility counts that
// gs_decode keeps in the caller's workspace) lives in one file-scope device
// array of kScratchInts int32 (512 KiB).  Every GPU on which the library is
// loaded holds that array until the process exits.
//
// Limits and sharing: the scratch holds ceil(N / 2048) * V counts, so calls
// with more than that are rejected on the host with GS_ERR_CAPACITY and
// nothing is enqueued.  All calls on a device share the one array: calls that
// overlap on the GPU (different streams or threads without ordering between
// them) race on it.  The counts are fully written before they are read, so
// nothing in the array has to start at zero and the contents a previous call
// left behind do not matter.
#include <mutex>

#include "gs_internal.cuh"

namespace {

constexpr int kScratchInts = 131072;   // 512 KiB of int32 counts
constexpr int kChunkAnchors = 2048;     // anchors per visibility block (as in decode.cu)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) int g_decode_scratch[kScratchInts];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of the array is only a stand-in).
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_decode_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GS_OK;
}

}  // namespace

extern "C" int gs_decode_noalloc(const gs_anchors *A, const gs_camera *cams, const gs_view *views, int32_t V,
                                 int32_t precision, gs_gauss3d *out, gs_status *status, void *stream)
{
    gs::ViewTable vt;
    if (!A || A->N < 0 || A->F < 1 || A->F > 64 || A->k < 1 || A->k > 16 || A->hidden < 1 || A->hidden > 64 ||
        A->M < 1 || (A->N > 0 && (!A->xyz || !A->feat || !A->log_scaling || !A->offsets || !A->part || !A->mlp)))
        return GS_ERR_INVALID_ARG;
    if (!cams || !status || !out || out->k != A->k || out->cap_rows < 0 || !out->row_anchor || !out->view_start ||
        !out->mu || !out->scale || !out->quat || !out->opacity || !out->colour ||
        out->cap_rows * (long long)out->k >= (1ll << 31) || !gs::make_view_table(views, V, &vt))
        return GS_ERR_INVALID_ARG;
    if (precision != GS_PREC_FP32 && precision != GS_PREC_BF16) return GS_ERR_INVALID_ARG;
    const long long counts = (long long)((A->N + kChunkAnchors - 1) / kChunkAnchors) * V;
    if (counts > kScratchInts) return GS_ERR_CAPACITY;
    if (gs::decode_workspace_bytes(A->N, V) > sizeof(int) * (size_t)kScratchInts) return GS_ERR_CAPACITY;
    void *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != GS_OK) return rc;
    return gs::launch_decode(A, cams, vt, precision, out, scratch, status, (cudaStream_t)stream);
}
