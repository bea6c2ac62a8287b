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

// Device address of the scratch array on the current device, looked up once per device (the first
// call on a device does the look-up).
int scratch_address(void **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(NM_ERR_ARG, "device ordinal %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(NM_ERR_CUDA, "cudaGetSymbolAddress of the staging array failed: %s", cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return NM_OK;
}

}  // namespace

extern "C" int nm_get_state_noalloc(nm_mesh M, double *m_out, double *t, double *dt)
{
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
