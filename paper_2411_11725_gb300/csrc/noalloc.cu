// nm_get_state_noalloc: nm_get_state into host memory without any allocation at call time.
//
// nm_get_state stages the node-major (AoS) copy of m in a stream-ordered device allocation before the
// device->host copy.  Callers that cannot allocate device memory at that point use this variant: a
// request loop that has committed its whole HBM budget to resident runs, or a caller that keeps
// allocator calls (which may synchronise or fail under memory pressure) out of its read-back path.
// Here the staging buffer is a fixed file-scope device array of kNoallocScratchBytes; meshes with more
// nodes than fit are rejected.
#include <mutex>

#include "mesh.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(4) << 20;  // 4 MiB: up to 174762 nodes (3 doubles each)
constexpr int kMaxDevices = 64;

// Staging for the AoS copy of m.  Nothing in it has to start at zero: the conversion kernel writes
// every element that the following device->host copy reads.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // id of the context the address belongs to

// The context id (cuCtxGetId, unique for the life of the process) tells whether the device's primary
// context is still the one the address was looked up in: after a cudaDeviceReset the module is loaded
// again and the array may sit elsewhere.  The two driver calls are reached through the runtime's
// entry-point query, so the library does not link the driver library directly.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_entry_once;

int current_context_id(unsigned long long *id)
{
    std::call_once(g_entry_once, [] {
        void *f = nullptr, *h = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &h, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            g_ctx_get_current = (CtxGetCurrentFn)f;
            g_ctx_get_id = (CtxGetIdFn)h;
        }
        cudaGetLastError();
    });
    if (!g_ctx_get_current || !g_ctx_get_id) return fail(NM_ERR_CUDA, "driver context queries unavailable");
    void *ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return fail(NM_ERR_CUDA, "no current CUDA context");
    if (g_ctx_get_id(ctx, id) != 0) return fail(NM_ERR_CUDA, "context id query failed");
    return NM_OK;
}

// Device address of the scratch array on the current device, looked up once per device and context
// (the first call on a device, and the first call after a reset of its primary context, do the
// look-up).
int scratch_address(void **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(NM_ERR_ARG, "device ordinal %d beyond %d", dev, kMaxDevices);
    CUDA_TRY(cudaSetDevice(dev));  // makes the device's primary context current on this thread
    unsigned long long ctx = 0;
    int rc = current_context_id(&ctx);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(NM_ERR_CUDA, "cudaGetSymbolAddress of the staging array failed: %s", cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return NM_OK;
}

}  // namespace

extern "C" int nm_get_state_noalloc(nm_mesh M, double *m_out, double *t, double *dt)
{
    clear_error();
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    const Geom &g = M->g;
    const size_t bytes = (size_t)g.n_nodes * 3 * sizeof(double);
    if (bytes > kNoallocScratchBytes)
        return fail(NM_ERR_ARG, "mesh has %ld nodes; nm_get_state_noalloc supports at most %ld", g.n_nodes,
                    (long)(kNoallocScratchBytes / (3 * sizeof(double))));
    if (!M->state_set) return fail(NM_ERR_STATE, "no state set");
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    if (m_out) {
        launch_soa_to_aos<double, double>(g, M->m, (double *)scratch, M->st);
        CHECK_LAUNCH();
        CUDA_TRY(cudaMemcpyAsync(m_out, scratch, bytes, cudaMemcpyDeviceToHost, M->st));
    }
    // waits for the copy: the staging array is free again when this returns
    if ((rc = pull_ctl(M))) return rc;
    if (t) *t = M->hctl->t;
    if (dt) *dt = M->hctl->dt;
    return NM_OK;
}
