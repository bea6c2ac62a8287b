// C ABI of the library (include/nmgb.h): mesh objects, device workspaces, argument validation, the
// Runge-Kutta step sequences and their CUDA-graph replay.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "mesh.cuh"

static thread_local std::string g_last_error;

void clear_error() { g_last_error.clear(); }

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

// --------------------------------------------------------------------------------------------- geometry
static int pad_len(int n)
{
    if (n == 1) return 1;
    int p = 1;
    while (p < 2 * n - 1) p *= 2;
    return p;
}
static int ilog2i(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

static Geom make_geom(int n1, int n2, int n3, int basis = 3)
{
    Geom g{};
    g.N1 = n1; g.N2 = n2; g.N3 = n3;
    g.basis = basis;
    g.nn1 = n1 + 1; g.nn2 = basis == 1 ? 1 : n2 + 1; g.nn3 = basis == 3 ? n3 + 1 : 1;
    g.zsn = basis == 3 ? g.nn1 * g.nn2 : 0;
    g.ysn = basis == 1 ? 0 : g.nn1;
    g.n_nodes = (long)g.nn1 * g.nn2 * g.nn3;
    g.n_cells = (long)n1 * n2 * n3;
    g.ns = round_up(g.n_nodes, 64);
    g.cs = round_up(g.n_cells, 64);
    g.P1 = pad_len(n1); g.P2 = pad_len(n2); g.P3 = pad_len(n3);
    g.Q = g.P1 == 1 ? 0 : g.P1 / 2;
    g.lgQ = g.Q ? ilog2i(g.Q) : 0;
    g.lgP2 = ilog2i(g.P2);
    g.lgP3 = ilog2i(g.P3);
    g.X = g.P1 / 2 + 1;
    g.Xp = (int)round_up(g.X, 16);
    g.H2 = g.P2 / 2 + 1;
    g.H3 = g.P3 / 2 + 1;
    int mx = g.P1 > g.P2 ? g.P1 : g.P2;
    mx = mx > g.P3 ? mx : g.P3;
    mx = mx < 4 ? 4 : mx;
    g.twlg = ilog2i(mx);
    g.s_comp = (long)n3 * g.P2 * g.Xp;
    g.t_comp = (long)g.H3 * g.H2 * g.Xp;
    g.n2f = FastDiv((unsigned)n2);
    return g;
}

static long footprint(const Geom &g, int prec)
{
    long rs = prec == NM_F64 ? 8 : 4;
    long b = 0;
    b += 3 * g.ns * 8;            // m
    if (prec == NM_F32) b += 3 * g.ns * 4;  // FP32 copy of m
    b += 2 * 3 * g.ns * rs;       // y ping-pong
    b += 7 * 3 * g.ns * rs;       // k1..k7
    b += 2 * 3 * g.ns * rs;       // h_eff in/out staging
    b += 2 * g.ns * rs;           // inv_mass, vol
    b += 3 * g.cs * rs;           // MsH
    b += 3 * g.s_comp * 2 * rs;   // spectra
    b += 6 * g.t_comp * rs;       // tensor spectrum
    b += 3 * g.cs * rs + 2 * g.cs * 8 + 3 * g.cs * 8;  // material maps (upper bound)
    return b;
}

template <typename T>
static void fill_twiddles(int twlg, std::vector<Cx<T>> &tw)
{
    const int n = 1 << twlg;
    tw.resize(n);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = 0; k < n; ++k) {
        long double a = -2.0L * pi * k / n;
        tw[k] = cx<T>((T)cosl(a), (T)sinl(a));
    }
}

// Device address of page-locked host memory that kernels may access directly, or NULL (pageable
// memory, or memory the current device cannot map).
void *mapped_host(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int can_map = 0, unified = 0;
    cudaDeviceGetAttribute(&can_map, cudaDevAttrCanMapHostMemory, dev);
    cudaDeviceGetAttribute(&unified, cudaDevAttrUnifiedAddressing, dev);
    if (!can_map || !unified) return nullptr;
    return a.devicePointer;
}

int dev_alloc(nm_mesh M, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NM_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    M->bytes += (long)bytes;
    return NM_OK;
}

void free_graphs(nm_mesh M)
{
    for (auto &gx : M->graph)
        if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
}

static void release(nm_mesh M)
{
    if (!M) return;
    cudaStreamSynchronize(M->st);
    free_graphs(M);
    void *ptrs[] = {M->m, M->mf, M->y[0], M->y[1], M->hin, M->hout, M->inv_mass, M->vol, M->MsH, M->S, M->Nk, M->tw,
                    M->tw64, M->A_d, M->Ku_d, M->Ms_d, M->Ms64_d, M->Msh_d, M->hcell64_d, M->D_d, M->hdmi, M->ctl,
                    M->partials,
                    M->mean_d, M->n_active_d, M->n_bad_d, M->vj_w, M->vj_h, M->vj_q, M->vj_g, M->vj_H, M->vj_HW, M->vj_M,
                    M->vj_gMs};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (void *p : M->k)
        if (p) cudaFree(p);
    for (void *p : M->extra)
        if (p) cudaFree(p);
    if (M->hctl) cudaFreeHost(M->hctl);
    if (M->mean_h) cudaFreeHost(M->mean_h);
    for (cudaEvent_t e : M->prof_ev) cudaEventDestroy(e);
    if (M->own_stream) cudaStreamDestroy(M->st);
    delete M;
}

long mesh_footprint(int n1, int n2, int n3, int precision)
{
    if (n1 < 1 || n2 < 1 || n3 < 1) return -1;
    return footprint(make_geom(n1, n2, n3), precision);
}

extern "C" long nm_footprint_bytes(int n1, int n2, int n3, int precision)
{
    return mesh_footprint(n1, n2, n3, precision);
}

extern "C" const char *nm_last_error(void) { return g_last_error.c_str(); }

extern "C" int nm_create_mesh(int n1, int n2, int n3, double dx1, double dx2, double dx3, int precision,
                              void *cuda_stream, nm_mesh *out)
{
    g_last_error.clear();
    return create_mesh(n1, n2, n3, dx1, dx2, dx3, precision, cuda_stream, nullptr, out);
}

extern "C" int nm_create_mesh_basis(int n1, int n2, int n3, double dx1, double dx2, double dx3, int precision,
                                    int basis, void *cuda_stream, nm_mesh *out)
{
    g_last_error.clear();
    if (basis < 1 || basis > 3) {
        if (out) *out = nullptr;
        return fail(NM_ERR_ARG, "basis must be 3 (trilinear), 2 (constant along z) or 1 (constant along y and z), got %d",
                    basis);
    }
    return create_mesh(n1, n2, n3, dx1, dx2, dx3, precision, cuda_stream, nullptr, out, basis);
}

int create_mesh(int n1, int n2, int n3, double dx1, double dx2, double dx3, int precision, void *cuda_stream,
                nm_mesh tensor_src, nm_mesh *out, int basis)
{
    if (!out) return fail(NM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n1 < 1 || n2 < 1 || n3 < 1) return fail(NM_ERR_ARG, "cell counts must be >= 1 (got %d %d %d)", n1, n2, n3);
    if (n1 > 1024 || n2 > 1024 || n3 > 64)
        return fail(NM_ERR_ARG, "grid %dx%dx%d beyond the supported range (N1, N2 <= 1024; N3 <= 64)", n1, n2, n3);
    if (!(dx1 > 0) || !(dx2 > 0) || !(dx3 > 0) || !isfinite(dx1) || !isfinite(dx2) || !isfinite(dx3))
        return fail(NM_ERR_ARG, "cell sizes must be positive and finite");
    if (precision != NM_F32 && precision != NM_F64) return fail(NM_ERR_ARG, "precision must be NM_F32 or NM_F64");
    {
        const Geom gg = make_geom(n1, n2, n3);
        const bool ok = precision == NM_F64 ? demag_plan<double>(gg).ok : demag_plan<float>(gg).ok;
        if (!ok)
            return fail(NM_ERR_ARG, "grid %dx%dx%d exceeds the FFT block budget of this precision", n1, n2, n3);
    }
    nm_mesh M = new nm_mesh_s();
    M->prec = precision;
    M->rs = precision == NM_F64 ? 8 : 4;
    M->g = make_geom(n1, n2, n3, basis);
    M->dx[0] = dx1; M->dx[1] = dx2; M->dx[2] = dx3;
    if (cuda_stream) {
        M->st = (cudaStream_t)cuda_stream;
        M->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&M->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete M;
            return fail(NM_ERR_CUDA, "cudaStreamCreate failed");
        }
        M->own_stream = true;
    }
    const Geom &g = M->g;
    const size_t rs = M->rs;
    int rc = NM_OK;
    demag_init_attributes();
#define ALLOC(p, b)                                      \
    if ((rc = dev_alloc(M, (void **)&(p), (b))) != NM_OK) { \
        release(M);                                      \
        return rc;                                       \
    }
    ALLOC(M->m, 3 * g.ns * 8);
    if (precision == NM_F32) ALLOC(M->mf, 3 * g.ns * 4);
    ALLOC(M->y[0], 3 * g.ns * rs);
    ALLOC(M->y[1], 3 * g.ns * rs);
    for (int i = 0; i < 7; ++i) ALLOC(M->k[i], 3 * g.ns * rs);
    ALLOC(M->hin, 3 * g.ns * rs);
    ALLOC(M->hout, 3 * g.ns * rs);
    ALLOC(M->inv_mass, g.ns * rs);
    ALLOC(M->vol, g.ns * rs);
    ALLOC(M->MsH, 3 * g.cs * rs);
    ALLOC(M->S, 3 * g.s_comp * 2 * rs);
    ALLOC(M->Nk, 6 * g.t_comp * rs);
    ALLOC(M->tw, (size_t)(1 << g.twlg) * 2 * rs);
    ALLOC(M->tw64, (size_t)(1 << g.twlg) * sizeof(Cx<double>));
    ALLOC(M->ctl, sizeof(StepCtl));
    ALLOC(M->partials, 4 * 1024 * sizeof(double));
    ALLOC(M->mean_d, 4 * sizeof(double));
    ALLOC(M->n_active_d, sizeof(unsigned long long));
    ALLOC(M->n_bad_d, sizeof(unsigned long long));
#undef ALLOC
    {
        const int er = precision == NM_F64 ? demag_encode_ymap<double>(g, M->S, &M->ymap)
                                           : demag_encode_ymap<float>(g, M->S, &M->ymap);
        if (er != 0) {
            release(M);
            return fail(NM_ERR_CUDA, "TMA descriptor of the inverse y pass refused (code %d)", er);
        }
    }
    if (cudaMallocHost(&M->hctl, sizeof(StepCtl)) != cudaSuccess ||
        cudaMallocHost(&M->mean_h, 4 * sizeof(double)) != cudaSuccess) {
        release(M);
        return fail(NM_ERR_OOM, "pinned host allocation failed");
    }
    memset(M->hctl, 0, sizeof(StepCtl));
    // zero everything that pads or may be read before written
    cudaMemsetAsync(M->m, 0, 3 * g.ns * 8, M->st);
    cudaMemsetAsync(M->y[0], 0, 3 * g.ns * rs, M->st);
    cudaMemsetAsync(M->y[1], 0, 3 * g.ns * rs, M->st);
    for (int i = 0; i < 7; ++i) cudaMemsetAsync(M->k[i], 0, 3 * g.ns * rs, M->st);
    cudaMemsetAsync(M->S, 0, 3 * g.s_comp * 2 * rs, M->st);
    cudaMemsetAsync(M->MsH, 0, 3 * g.cs * rs, M->st);
    cudaMemsetAsync(M->ctl, 0, sizeof(StepCtl), M->st);
    cudaError_t e;
    if (tensor_src && tensor_src->prec == precision && tensor_src->g.P1 == g.P1 && tensor_src->g.P2 == g.P2 &&
        tensor_src->g.P3 == g.P3 && tensor_src->g.N1 == n1 && tensor_src->g.N2 == n2 && tensor_src->g.N3 == n3 &&
        tensor_src->dx[0] == dx1 && tensor_src->dx[1] == dx2 && tensor_src->dx[2] == dx3) {
        // same shape, cell size and precision: the twiddles and the tensor spectrum are copied, not rebuilt
        cudaMemcpyAsync(M->tw64, tensor_src->tw64, (size_t)(1 << g.twlg) * sizeof(Cx<double>),
                        cudaMemcpyDeviceToDevice, M->st);
        cudaMemcpyAsync(M->tw, tensor_src->tw, (size_t)(1 << g.twlg) * 2 * rs, cudaMemcpyDeviceToDevice, M->st);
        cudaMemcpyAsync(M->Nk, tensor_src->Nk, 6 * g.t_comp * rs, cudaMemcpyDeviceToDevice, M->st);
        e = cudaStreamSynchronize(M->st);
        if (e != cudaSuccess) {
            release(M);
            return fail(NM_ERR_CUDA, "mesh set-up failed: %s", cudaGetErrorString(e));
        }
        *out = M;
        return NM_OK;
    }
    // twiddles (host, long double) and the tensor spectrum (device, FP64)
    std::vector<Cx<double>> tw64;
    fill_twiddles<double>(g.twlg, tw64);
    cudaMemcpyAsync(M->tw64, tw64.data(), tw64.size() * sizeof(Cx<double>), cudaMemcpyHostToDevice, M->st);
    if (precision == NM_F64) {
        cudaMemcpyAsync(M->tw, tw64.data(), tw64.size() * sizeof(Cx<double>), cudaMemcpyHostToDevice, M->st);
        e = build_tensor_spectrum<double>(g, dx1, dx2, dx3, M->tw64, (double *)M->Nk, M->st);
    } else {
        std::vector<Cx<float>> tw32;
        fill_twiddles<float>(g.twlg, tw32);
        cudaMemcpyAsync(M->tw, tw32.data(), tw32.size() * sizeof(Cx<float>), cudaMemcpyHostToDevice, M->st);
        e = build_tensor_spectrum<float>(g, dx1, dx2, dx3, M->tw64, (float *)M->Nk, M->st);
        cudaStreamSynchronize(M->st);  // tw32 goes out of scope
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->st);
    if (e != cudaSuccess) {
        release(M);
        return fail(NM_ERR_CUDA, "mesh set-up failed: %s", cudaGetErrorString(e));
    }
    *out = M;
    return NM_OK;
}

extern "C" int nm_destroy_mesh(nm_mesh M)
{
    release(M);
    return NM_OK;
}

extern "C" int nm_mesh_info(nm_mesh M, long *n_nodes, long *n_cells, int P[3], long *device_bytes)
{
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (n_nodes) *n_nodes = M->g.n_nodes;
    if (n_cells) *n_cells = M->g.n_cells;
    if (P) { P[0] = M->g.P1; P[1] = M->g.P2; P[2] = M->g.P3; }
    if (device_bytes) *device_bytes = M->bytes;
    return NM_OK;
}

extern "C" int nm_sync(nm_mesh M)
{
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    CUDA_TRY(cudaStreamSynchronize(M->st));
    return NM_OK;
}

// --------------------------------------------------------------------------------------------- material
static bool all_finite(const double *a, long n, double *mn)
{
    double lo = INFINITY;
    for (long i = 0; i < n; ++i) {
        if (!isfinite(a[i])) return false;
        lo = a[i] < lo ? a[i] : lo;
    }
    *mn = lo;
    return true;
}

// host cell array (c1 slowest) -> device internal layout (c1 fastest) in type T
template <typename T>
static int upload_cells(nm_mesh M, const double *h, int ncomp, void **dst, bool want_double, double **dst64)
{
    const Geom &g = M->g;
    double *tmp = nullptr;
    CUDA_TRY(cudaMallocAsync(&tmp, g.n_cells * ncomp * sizeof(double), M->st));
    CUDA_TRY(cudaMemcpyAsync(tmp, h, g.n_cells * ncomp * sizeof(double), cudaMemcpyHostToDevice, M->st));
    if (dst) {
        if (!*dst) {
            int rc = dev_alloc(M, dst, ncomp * g.cs * sizeof(T));
            if (rc) return rc;
        }
        launch_cells_to_internal<T>(g, tmp, ncomp, 0.0, nullptr, (T *)*dst, M->st);
    }
    if (want_double) {
        if (!*dst64) {
            int rc = dev_alloc(M, (void **)dst64, ncomp * g.cs * sizeof(double));
            if (rc) return rc;
        }
        launch_cells_to_internal<double>(g, tmp, ncomp, 0.0, nullptr, *dst64, M->st);
    }
    CHECK_LAUNCH();
    CUDA_TRY(cudaFreeAsync(tmp, M->st));
    return NM_OK;
}

template <typename T>
static int set_material_t(nm_mesh M, const double *Ms, const double *A, const double *Ku)
{
    const Geom &g = M->g;
    int rc;
    if (Ms) {
        if ((rc = upload_cells<T>(M, Ms, 1, &M->Ms_d, true, &M->Ms64_d))) return rc;
    } else {
        if (M->Ms_d) { cudaFree(M->Ms_d); M->Ms_d = nullptr; }
        if (M->Ms64_d) { cudaFree(M->Ms64_d); M->Ms64_d = nullptr; }
    }
    if (A) {
        if ((rc = upload_cells<T>(M, A, 1, &M->A_d, false, nullptr))) return rc;
    } else if (M->A_d) { cudaFree(M->A_d); M->A_d = nullptr; }
    if (Ku) {
        if ((rc = upload_cells<T>(M, Ku, 1, &M->Ku_d, false, nullptr))) return rc;
    } else if (M->Ku_d) { cudaFree(M->Ku_d); M->Ku_d = nullptr; }
    CUDA_TRY(cudaMemsetAsync(M->n_active_d, 0, sizeof(unsigned long long), M->st));
    const double V = M->dx[0] * M->dx[1] * M->dx[2];
    launch_mass<T>(g, M->Ms64_d, M->Ms0, V, (T *)M->inv_mass, M->n_active_d, M->st);
    launch_node_volume<T>(g, M->Ms64_d, M->Ms0, V, (T *)M->vol, M->st);
    CHECK_LAUNCH();
    unsigned long long na = 0;
    CUDA_TRY(cudaMemcpyAsync(&na, M->n_active_d, sizeof na, cudaMemcpyDeviceToHost, M->st));
    CUDA_TRY(cudaStreamSynchronize(M->st));
    M->n_active = (double)na;
    return NM_OK;
}

static int rebuild_cell_field(nm_mesh M);

template <typename T>
static int set_dmi_t(nm_mesh M, const double *D)
{
    int rc;
    if (D) {
        if ((rc = upload_cells<T>(M, D, 1, &M->D_d, false, nullptr))) return rc;
    } else if (M->D_d) {
        cudaFree(M->D_d);
        M->D_d = nullptr;
    }
    if (!M->hdmi && (rc = dev_alloc(M, &M->hdmi, 3 * M->g.ns * sizeof(T)))) return rc;
    CUDA_TRY(cudaMemsetAsync(M->hdmi, 0, 3 * M->g.ns * sizeof(T), M->st));
    return NM_OK;
}

extern "C" int nm_set_dmi(nm_mesh M, const double *D, double D0)
{
    g_last_error.clear();
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (M->g.basis != 3) return fail(NM_ERR_ARG, "the DMI term needs the 3D nodal basis");
    double mn;
    if (D && !all_finite(D, M->g.n_cells, &mn)) return fail(NM_ERR_ARG, "D map must be finite");
    if (!D && !isfinite(D0)) return fail(NM_ERR_ARG, "D0 must be finite");
    free_graphs(M);
    int rc = M->prec == NM_F64 ? set_dmi_t<double>(M, D) : set_dmi_t<float>(M, D);
    if (rc) return rc;
    M->D0 = D ? 0.0 : D0;
    M->has_dmi = true;
    M->k1_valid = false;
    return NM_OK;
}

extern "C" int nm_set_material(nm_mesh M, const double *Ms, double Ms0, const double *A, double A0,
                               const double *Ku, double Ku0, const double axis[3], double alpha, double gamma)
{
    g_last_error.clear();
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (!axis) return fail(NM_ERR_ARG, "axis is NULL");
    double an = sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    if (!(an > 0) || !isfinite(an)) return fail(NM_ERR_ARG, "axis must be a non-zero finite vector");
    if (!isfinite(alpha) || alpha < 0 || !isfinite(gamma)) return fail(NM_ERR_ARG, "alpha/gamma invalid");
    const long nc = M->g.n_cells;
    double mn;
    if (Ms && (!all_finite(Ms, nc, &mn) || mn < 0)) return fail(NM_ERR_ARG, "Ms map must be finite and >= 0");
    if (!Ms && (!isfinite(Ms0) || Ms0 < 0)) return fail(NM_ERR_ARG, "Ms0 must be finite and >= 0");
    if (A && !all_finite(A, nc, &mn)) return fail(NM_ERR_ARG, "A map must be finite");
    if (Ku && !all_finite(Ku, nc, &mn)) return fail(NM_ERR_ARG, "Ku map must be finite");
    if (!isfinite(A0) || !isfinite(Ku0)) return fail(NM_ERR_ARG, "A0/Ku0 must be finite");
    M->Ms0 = Ms ? 0.0 : Ms0;
    M->A0 = A0;
    M->Ku0 = Ku0;
    for (int k = 0; k < 3; ++k) M->axis[k] = axis[k] / an;
    M->alpha = alpha;
    M->gamma = gamma;
    free_graphs(M);
    int rc = M->prec == NM_F64 ? set_material_t<double>(M, Ms, A, Ku) : set_material_t<float>(M, Ms, A, Ku);
    if (rc) return rc;
    M->material_set = true;
    M->k1_valid = false;
    return rebuild_cell_field(M);
}

// Ms_c h_c for the cell applied field
template <typename T>
__global__ void k_ms_times(long nc, long cs, const double *__restrict__ h, const double *__restrict__ Ms, double Ms0,
                           T *__restrict__ out)
{
    long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double ms = Ms ? Ms[c] : Ms0;
    for (int j = 0; j < 3; ++j) out[j * cs + c] = (T)(ms * h[j * cs + c]);
}

static int rebuild_cell_field(nm_mesh M)
{
    if (!M->has_hcell || !M->material_set) return NM_OK;
    const Geom &g = M->g;
    if (!M->Msh_d) {
        int rc = dev_alloc(M, &M->Msh_d, 3 * g.cs * M->rs);
        if (rc) return rc;
    }
    if (M->prec == NM_F64)
        k_ms_times<double><<<div_up(g.n_cells, 256), 256, 0, M->st>>>(g.n_cells, g.cs, M->hcell64_d, M->Ms64_d, M->Ms0,
                                                                      (double *)M->Msh_d);
    else
        k_ms_times<float><<<div_up(g.n_cells, 256), 256, 0, M->st>>>(g.n_cells, g.cs, M->hcell64_d, M->Ms64_d, M->Ms0,
                                                                     (float *)M->Msh_d);
    CHECK_LAUNCH();
    return NM_OK;
}

extern "C" int nm_set_field(nm_mesh M, int kind, const double *data, const double amp[3], double freq_hz,
                            double phase)
{
    g_last_error.clear();
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (!isfinite(freq_hz) || !isfinite(phase)) return fail(NM_ERR_ARG, "freq/phase must be finite");
    free_graphs(M);
    if (kind == NM_FIELD_HEXT_UNIFORM) {
        if (!amp) return fail(NM_ERR_ARG, "amp is NULL");
        for (int k = 0; k < 3; ++k) {
            if (!isfinite(amp[k])) return fail(NM_ERR_ARG, "amp must be finite");
            M->hu[k] = amp[k];
        }
        M->hu_freq = freq_hz;
        M->hu_phase = phase;
        return NM_OK;
    }
    if (kind == NM_FIELD_HEXT_CELL) {
        M->hc_freq = freq_hz;
        M->hc_phase = phase;
        if (!data) {
            M->has_hcell = false;
            return NM_OK;
        }
        double mn;
        if (!all_finite(data, 3 * M->g.n_cells, &mn)) return fail(NM_ERR_ARG, "cell field must be finite");
        int rc = upload_cells<double>(M, data, 3, nullptr, true, &M->hcell64_d);
        if (rc) return rc;
        M->has_hcell = true;
        return rebuild_cell_field(M);
    }
    return fail(NM_ERR_ARG, "unknown field kind %d", kind);
}

extern "C" int nm_set_terms(nm_mesh M, unsigned terms)
{
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (terms & ~NM_TERMS_MASK) return fail(NM_ERR_ARG, "unknown term bits 0x%x", terms);
    M->terms = terms;
    M->k1_valid = false;
    free_graphs(M);
    return NM_OK;
}

extern "C" int nm_set_error_norm(nm_mesh M, int fp64_terms)
{
    g_last_error.clear();
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    M->err_f64_terms = fp64_terms ? 1 : 0;
    free_graphs(M);
    return NM_OK;
}

extern "C" int nm_set_integrator(nm_mesh M, int renormalise, double dt_min, int max_rejections)
{
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (!(dt_min >= 0) || max_rejections < 1) return fail(NM_ERR_ARG, "dt_min >= 0 and max_rejections >= 1");
    M->renorm = renormalise ? 1 : 0;
    M->dt_min = dt_min;
    M->max_rej = max_rejections;
    free_graphs(M);
    return NM_OK;
}

// --------------------------------------------------------------------------------------------- state
extern "C" int nm_set_state(nm_mesh M, const double *m, int where, double t, double dt)
{
    g_last_error.clear();
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (!m) return fail(NM_ERR_ARG, "m is NULL");
    if (where != NM_MEM_HOST && where != NM_MEM_DEVICE) return fail(NM_ERR_ARG, "where must be host or device");
    if (!isfinite(t) || !isfinite(dt)) return fail(NM_ERR_ARG, "t/dt must be finite");
    const Geom &g = M->g;
    const double *src = m;
    double *tmp = nullptr;
    if (where == NM_MEM_HOST) {
        const void *mapped = mapped_host(m);
        if (mapped) {
            src = (const double *)mapped;  // page-locked: the conversion reads it over the link directly
        } else {
            CUDA_TRY(cudaMallocAsync(&tmp, g.n_nodes * 3 * sizeof(double), M->st));
            CUDA_TRY(cudaMemcpyAsync(tmp, m, g.n_nodes * 3 * sizeof(double), cudaMemcpyHostToDevice, M->st));
            src = tmp;
        }
    }
    CUDA_TRY(cudaMemsetAsync(M->n_bad_d, 0, sizeof(unsigned long long), M->st));
    launch_aos_to_soa<double, double>(g, src, M->m, M->st, M->n_bad_d);
    CHECK_LAUNCH();
    if (tmp) CUDA_TRY(cudaFreeAsync(tmp, M->st));
    unsigned long long n_bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&n_bad, M->n_bad_d, sizeof n_bad, cudaMemcpyDeviceToHost, M->st));
    StepCtl *h = M->hctl;
    CUDA_TRY(cudaStreamSynchronize(M->st));
    M->k1_valid = false;
    M->mf_valid = false;
    if (n_bad) {
        // the resident m now holds the rejected values: no integration until a valid state is set
        M->state_set = false;
        return fail(NM_ERR_NONFINITE, "m holds non-finite values at %llu nodes; state not set", n_bad);
    }
    memset(h, 0, sizeof(StepCtl));
    h->t = t;
    h->dt = dt;
    h->dt_min = M->dt_min;
    CUDA_TRY(cudaMemcpyAsync(M->ctl, h, sizeof(StepCtl), cudaMemcpyHostToDevice, M->st));
    M->state_set = true;
    M->k1_valid = false;
    M->mf_valid = false;
    return NM_OK;
}

int ensure_mf(nm_mesh M)
{
    if (!M->mf || M->mf_valid) return NM_OK;
    launch_convert<double, float>(3 * M->g.ns, M->m, M->mf, M->st);
    CHECK_LAUNCH();
    M->mf_valid = true;
    return NM_OK;
}

int pull_ctl(nm_mesh M)
{
    CUDA_TRY(cudaMemcpyAsync(M->hctl, M->ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, M->st));
    CUDA_TRY(cudaStreamSynchronize(M->st));
    return NM_OK;
}
int push_ctl(nm_mesh M)
{
    CUDA_TRY(cudaMemcpyAsync(M->ctl, M->hctl, sizeof(StepCtl), cudaMemcpyHostToDevice, M->st));
    return NM_OK;
}

extern "C" int nm_get_state(nm_mesh M, double *m_out, int where, double *t, double *dt)
{
    g_last_error.clear();
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (!M->state_set) return fail(NM_ERR_STATE, "no state set");
    if (where != NM_MEM_HOST && where != NM_MEM_DEVICE) return fail(NM_ERR_ARG, "where must be host or device");
    const Geom &g = M->g;
    if (m_out) {
        if (where == NM_MEM_DEVICE) {
            launch_soa_to_aos<double, double>(g, M->m, m_out, M->st);
            CHECK_LAUNCH();
        } else if (void *mapped = mapped_host(m_out)) {
            // page-locked: the conversion writes it over the link directly
            launch_soa_to_aos<double, double>(g, M->m, (double *)mapped, M->st);
            CHECK_LAUNCH();
        } else {
            double *tmp = nullptr;
            CUDA_TRY(cudaMallocAsync(&tmp, g.n_nodes * 3 * sizeof(double), M->st));
            launch_soa_to_aos<double, double>(g, M->m, tmp, M->st);
            CHECK_LAUNCH();
            CUDA_TRY(cudaMemcpyAsync(m_out, tmp, g.n_nodes * 3 * sizeof(double), cudaMemcpyDeviceToHost, M->st));
            CUDA_TRY(cudaFreeAsync(tmp, M->st));
        }
    }
    int rc = pull_ctl(M);
    if (rc) return rc;
    if (t) *t = M->hctl->t;
    if (dt) *dt = M->hctl->dt;
    return NM_OK;
}

extern "C" int nm_get_counters(nm_mesh M, long *n_accepted, long *n_rejected, double *last_err)
{
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    int rc = pull_ctl(M);
    if (rc) return rc;
    if (n_accepted) *n_accepted = M->hctl->n_acc;
    if (n_rejected) *n_rejected = M->hctl->n_rej;
    if (last_err) *last_err = M->hctl->err;
    return NM_OK;
}

// --------------------------------------------------------------------------------------------- field pipeline
template <typename T>
static int heff_t(nm_mesh M, const void *m, void *h_out, unsigned terms, double t)
{
    const Geom &g = M->g;
    if (m) launch_aos_to_soa<T, T>(g, (const T *)m, (T *)M->hin, M->st);
    else launch_convert<double, T>(3 * g.ns, M->m, (T *)M->hin, M->st);
    if (terms & NM_DEMAG) demag_forward<T>(g, demag_bufs<T>(M), (const T *)M->hin, (T *)M->MsH, M->st);
    launch_heff<T>(local_params<T>(M, terms), (const T *)M->hin, (T *)M->hout, t, M->st);
    launch_soa_to_aos<T, T>(g, (const T *)M->hout, (T *)h_out, M->st);
    CHECK_LAUNCH();
    return NM_OK;
}

extern "C" int nm_h_eff(nm_mesh M, const void *m, void *h_out, unsigned terms, double t)
{
    g_last_error.clear();
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (!h_out) return fail(NM_ERR_ARG, "h_out is NULL");
    if (terms & ~NM_TERMS_MASK) return fail(NM_ERR_ARG, "unknown term bits 0x%x", terms);
    if (!isfinite(t)) return fail(NM_ERR_ARG, "t must be finite");
    if (!M->material_set) return fail(NM_ERR_STATE, "material not set");
    if (!m && !M->state_set) return fail(NM_ERR_STATE, "m is NULL and no resident state");
    return M->prec == NM_F64 ? heff_t<double>(M, m, h_out, terms, t) : heff_t<float>(M, m, h_out, terms, t);
}

// --------------------------------------------------------------------------------------------- RK steps
// slope of stage s from input y_s; optionally the next stage input from the tableau row a_next
template <typename T>
static void enqueue_stage(nm_mesh M, const LocalParams<T> &p, int s, double c_s, const T *ys, T *ynext,
                          const double *a_next, int n_next)
{
    const Geom &g = M->g;
    if (p.terms & NM_DEMAG) {
        DemagBufs<T> b = demag_bufs<T>(M);
        b.ctl = M->ctl;
        demag_forward<T>(g, b, ys, (T *)M->MsH, M->st);
    }
    StageArgs sa{};
    sa.m = M->m;
    sa.mf = M->mf;
    for (int j = 0; j < 7; ++j) sa.k[j] = M->k[j];
    for (int j = 0; j < n_next; ++j) {
        sa.a[j] = a_next[j];
        sa.af[j] = (float)a_next[j];
    }
    sa.s = s;
    sa.a_s = n_next >= s ? a_next[s - 1] : 0.0;
    sa.af_s = (float)sa.a_s;
    sa.c_s = c_s;
    sa.ctl = M->ctl;
    launch_llg_stage<T>(p, ys, (T *)M->k[s - 1], ynext, sa, M->st);
    marker(M)("node_llg_stage");
}

// k1 = f(m) at the resident time (first DP5 step after a state change)
template <typename T>
static void enqueue_k1(nm_mesh M)
{
    const LocalParams<T> p = local_params<T>(M, M->terms);
    KList none{};
    launch_stage_input<T>(M->g, M->m, none, M->ctl, (T *)M->y[0], M->st, M->mf);
    enqueue_stage<T>(M, p, 1, 0.0, (const T *)M->y[0], nullptr, nullptr, 0);
}

template <typename T>
static void enqueue_dp5_step(nm_mesh M)
{
    const LocalParams<T> p = local_params<T>(M, M->terms);
    const Geom &g = M->g;
    KList k2in{};
    k2in.p[0] = M->k[0];
    k2in.a[0] = kDpA[1][0];
    k2in.n = 1;
    launch_stage_input<T>(g, M->m, k2in, M->ctl, (T *)M->y[0], M->st, M->mf);  // y_2
    marker(M)("stage_input");
    for (int s = 2; s <= 7; ++s) {
        const T *ys = (const T *)M->y[s % 2];
        T *yn = s < 7 ? (T *)M->y[(s + 1) % 2] : nullptr;
        enqueue_stage<T>(M, p, s, kDpC[s - 1], ys, yn, s < 7 ? kDpA[s] : nullptr, s < 7 ? s : 0);
    }
    KList kb{}, ke{};
    const int idx[6] = {0, 2, 3, 4, 5, 6};
    for (int j = 0; j < 6; ++j) {
        kb.p[j] = ke.p[j] = M->k[idx[j]];
        kb.a[j] = kDpB[idx[j]];
        ke.a[j] = kDpB[idx[j]] - kDpBs[idx[j]];
    }
    kb.n = ke.n = 6;
    launch_dp5_control<T>(g, M->m, kb, ke, (const T *)M->inv_mass, M->ctl, M->partials, M->n_active, M->max_rej,
                          M->st, M->mf, M->err_f64_terms != 0);
    marker(M)("dp5_error_control");
    KList ku = kb;
    ku.n = 5;  // b7 = 0
    launch_dp5_update<T>(g, M->m, ku, (const T *)M->k[6], (T *)M->k[0], M->ctl, M->renorm, M->st, M->mf);
    marker(M)("dp5_update");
}

template <typename T>
static void enqueue_rk4_step(nm_mesh M)
{
    const LocalParams<T> p = local_params<T>(M, M->terms);
    const Geom &g = M->g;
    KList none{};
    launch_stage_input<T>(g, M->m, none, M->ctl, (T *)M->y[1], M->st, M->mf);  // y_1 = m
    marker(M)("stage_input");
    for (int s = 1; s <= 4; ++s) {
        const T *ys = (const T *)M->y[s % 2];
        T *yn = s < 4 ? (T *)M->y[(s + 1) % 2] : nullptr;
        enqueue_stage<T>(M, p, s, kRk4C[s - 1], ys, yn, s < 4 ? kRk4A[s] : nullptr, s < 4 ? s : 0);
    }
    KList kb{};
    for (int j = 0; j < 4; ++j) {
        kb.p[j] = M->k[j];
        kb.a[j] = kRk4B[j];
    }
    kb.n = 4;
    launch_rk4_update<T>(g, M->m, kb, M->ctl, M->renorm, M->st, M->mf);
    marker(M)("rk4_update");
}

static int enqueue_step(nm_mesh M, int method)
{
    if (method == NM_DP54) {
        if (M->prec == NM_F64) enqueue_dp5_step<double>(M);
        else enqueue_dp5_step<float>(M);
    } else {
        if (M->prec == NM_F64) enqueue_rk4_step<double>(M);
        else enqueue_rk4_step<float>(M);
    }
    CHECK_LAUNCH();
    return NM_OK;
}

int launch_step(nm_mesh M, int method)
{
    int rc0 = ensure_mf(M);
    if (rc0) return rc0;
    cudaGraphExec_t &gx = M->graph[method];
    if (!gx) {
        cudaGraph_t graph;
        CUDA_TRY(cudaStreamBeginCapture(M->st, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_step(M, method);
        cudaError_t e = cudaStreamEndCapture(M->st, &graph);
        if (rc) return rc;
        if (e != cudaSuccess) return fail(NM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&gx, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            gx = nullptr;
            return fail(NM_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
        }
    }
    CUDA_TRY(cudaGraphLaunch(gx, M->st));
    return NM_OK;
}

int ensure_k1(nm_mesh M, int method)
{
    if (method != NM_DP54 || M->k1_valid) return NM_OK;
    int rc0 = ensure_mf(M);
    if (rc0) return rc0;
    if (M->prec == NM_F64) enqueue_k1<double>(M);
    else enqueue_k1<float>(M);
    CHECK_LAUNCH();
    M->k1_valid = true;
    return NM_OK;
}

int check_step_args(nm_mesh M, int method, double rtol, double atol)
{
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (method != NM_RK4 && method != NM_DP54) return fail(NM_ERR_ARG, "unknown method %d", method);
    if (method == NM_DP54 && (!(rtol >= 0) || !(atol >= 0) || (rtol == 0 && atol == 0) || !isfinite(rtol) ||
                              !isfinite(atol)))
        return fail(NM_ERR_ARG, "tolerances must be finite, >= 0 and not both 0");
    if (!M->material_set) return fail(NM_ERR_STATE, "material not set");
    if (!M->state_set) return fail(NM_ERR_STATE, "state not set");
    return NM_OK;
}

extern "C" int nm_llg_step(nm_mesh M, int method, double *t, double *dt, double rtol, double atol, int *accepted)
{
    g_last_error.clear();
    int rc = check_step_args(M, method, rtol, atol);
    if (rc) return rc;
    if (!t || !dt) return fail(NM_ERR_ARG, "t/dt NULL");
    if (!(*dt > 0) || !isfinite(*dt) || !isfinite(*t)) return fail(NM_ERR_ARG, "dt must be positive and finite");
    if ((rc = pull_ctl(M))) return rc;
    StepCtl *h = M->hctl;
    h->t = *t;
    h->dt = *dt;
    h->rtol = rtol;
    h->atol = atol;
    h->t_end = 0.0;
    h->done = 0;
    h->status = NM_OK;
    h->dt_min = M->dt_min;
    if ((rc = push_ctl(M))) return rc;
    if ((rc = ensure_k1(M, method))) return rc;
    if ((rc = launch_step(M, method))) return rc;
    if ((rc = pull_ctl(M))) return rc;
    *t = h->t;
    *dt = h->dt;
    if (accepted) *accepted = h->accepted;
    if (h->status != NM_OK) return fail(h->status, "step failed (status %d, err %g)", h->status, h->err);
    return NM_OK;
}

extern "C" int nm_run_steps(nm_mesh M, int method, long n_steps, double rtol, double atol)
{
    g_last_error.clear();
    int rc = check_step_args(M, method, rtol, atol);
    if (rc) return rc;
    if (n_steps < 0) return fail(NM_ERR_ARG, "n_steps < 0");
    if ((rc = pull_ctl(M))) return rc;
    StepCtl *h = M->hctl;
    if (!(h->dt > 0)) return fail(NM_ERR_STATE, "resident dt must be positive");
    h->rtol = rtol;
    h->atol = atol;
    h->t_end = 0.0;
    h->done = 0;
    h->status = NM_OK;
    h->dt_min = M->dt_min;
    if ((rc = push_ctl(M))) return rc;
    if ((rc = ensure_k1(M, method))) return rc;
    for (long i = 0; i < n_steps; ++i)
        if ((rc = launch_step(M, method))) return rc;
    return NM_OK;
}

template <typename T>
static void enqueue_mean(nm_mesh M)
{
    launch_mean<T>(M->g, M->m, (const T *)M->vol, M->partials, M->mean_d, M->st);
}

static int record_mean(nm_mesh M, double *out3)
{
    if (M->prec == NM_F64) enqueue_mean<double>(M);
    else enqueue_mean<float>(M);
    CHECK_LAUNCH();
    CUDA_TRY(cudaMemcpyAsync(M->mean_h, M->mean_d, 4 * sizeof(double), cudaMemcpyDeviceToHost, M->st));
    CUDA_TRY(cudaStreamSynchronize(M->st));
    for (int j = 0; j < 3; ++j) out3[j] = M->mean_h[j];
    return NM_OK;
}

extern "C" int nm_mean_m(nm_mesh M, double *out)
{
    g_last_error.clear();
    if (!M || !out) return fail(NM_ERR_ARG, "mesh and out are required");
    if (!M->state_set) return fail(NM_ERR_STATE, "no state set");
    return record_mean(M, out);
}

extern "C" int nm_run_until(nm_mesh M, double t_end, int method, double rtol, double atol, double dt0,
                            double sample_dt, double *samples_out, long max_samples, long *n_accepted,
                            long *n_rejected)
{
    g_last_error.clear();
    int rc = check_step_args(M, method, rtol, atol);
    if (rc) return rc;
    if (!isfinite(t_end) || !isfinite(dt0) || !isfinite(sample_dt)) return fail(NM_ERR_ARG, "non-finite argument");
    if (sample_dt > 0 && (!samples_out || max_samples < 1)) return fail(NM_ERR_ARG, "samples_out/max_samples");
    if ((rc = pull_ctl(M))) return rc;
    StepCtl *h = M->hctl;
    const double t0 = h->t;
    if (t_end < t0) return fail(NM_ERR_ARG, "t_end before the resident time");
    double dt = dt0 > 0 ? dt0 : h->dt;
    if (!(dt > 0)) return fail(NM_ERR_ARG, "no positive step size");
    const long acc0 = h->n_acc, rej0 = h->n_rej;
    long ks = 0;
    if (sample_dt > 0) {
        if ((rc = record_mean(M, samples_out))) return rc;
        ks = 1;
    }
    const double tiny = 1e-12 * (fabs(t_end) > 0 ? fabs(t_end) : 1.0);
    double t = t0;
    while (t < t_end - tiny) {
        double target = t_end;
        if (sample_dt > 0) {
            double ts = t0 + ks * sample_dt;
            if (ts < target) target = ts;
        }
        // integrate to target with the device clipping the step at target
        if ((rc = pull_ctl(M))) return rc;
        h->t = t;
        h->dt = method == NM_RK4 ? dt0 : dt;
        if (h->dt > target - t) h->dt = target - t;
        h->t_end = target;
        h->rtol = rtol;
        h->atol = atol;
        h->done = 0;
        h->status = NM_OK;
        h->dt_min = M->dt_min;
        if ((rc = push_ctl(M))) return rc;
        if ((rc = ensure_k1(M, method))) return rc;
        long chunk = 1;
        while (true) {
            for (long i = 0; i < chunk; ++i)
                if ((rc = launch_step(M, method))) return rc;
            if ((rc = pull_ctl(M))) return rc;
            if (h->status != NM_OK) return fail(h->status, "integration failed at t=%g (err %g)", h->t, h->err);
            if (h->done) break;
            if (chunk < 64) chunk *= 2;
        }
        t = h->t;
        if (method == NM_DP54) dt = h->dt_prop > 0 ? h->dt_prop : h->dt;
        if (sample_dt > 0 && fabs(t - (t0 + ks * sample_dt)) <= tiny + 1e-9 * sample_dt) {
            if (ks < max_samples && (rc = record_mean(M, samples_out + 3 * ks))) return rc;
            ++ks;
        }
    }
    if ((rc = pull_ctl(M))) return rc;
    h->t_end = 0.0;
    h->done = 0;
    h->dt = method == NM_DP54 ? dt : h->dt;
    if ((rc = push_ctl(M))) return rc;
    if (n_accepted) *n_accepted = h->n_acc - acc0;
    if (n_rejected) *n_rejected = h->n_rej - rej0;
    return NM_OK;
}

extern "C" int nm_profile_step(nm_mesh M, int method, int reps, double rtol, double atol, int max_kernels,
                               double *ms_out, char *names_out, int *n_kernels)
{
    g_last_error.clear();
    int rc = check_step_args(M, method, rtol, atol);
    if (rc) return rc;
    if (reps < 1 || max_kernels < 1 || !ms_out || !n_kernels) return fail(NM_ERR_ARG, "bad profiling arguments");
    if ((rc = pull_ctl(M))) return rc;
    StepCtl *h = M->hctl;
    h->rtol = rtol;
    h->atol = atol;
    h->t_end = 0.0;
    h->done = 0;
    h->status = NM_OK;
    if ((rc = push_ctl(M))) return rc;
    if ((rc = ensure_k1(M, method))) return rc;
    free_graphs(M);  // graphs hold no markers
    std::vector<double> acc;
    int nk = 0;
    cudaEvent_t start;
    CUDA_TRY(cudaEventCreate(&start));
    for (int r = 0; r < reps; ++r) {
        M->prof_on = true;
        M->prof_n = 0;
        cudaEventRecord(start, M->st);
        rc = enqueue_step(M, method);
        M->prof_on = false;
        if (rc) { cudaEventDestroy(start); return rc; }
        CUDA_TRY(cudaStreamSynchronize(M->st));
        nk = (int)M->prof_n;
        if (acc.empty()) acc.assign(nk, 0.0);
        cudaEvent_t prev = start;
        for (int i = 0; i < nk; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, prev, M->prof_ev[i]);
            acc[i] += ms;
            prev = M->prof_ev[i];
        }
    }
    cudaEventDestroy(start);
    *n_kernels = nk;
    for (int i = 0; i < nk && i < max_kernels; ++i) {
        ms_out[i] = acc[i] / reps;
        if (names_out) {
            strncpy(names_out + 32 * i, M->prof_names[i], 31);
            names_out[32 * i + 31] = 0;
        }
    }
    return NM_OK;
}
