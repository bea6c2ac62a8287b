// Mesh object shared by the library's translation units: device workspaces, model parameters and
// the helpers that assemble kernel parameter blocks from them.
#pragma once
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "local.cuh"
#include "newell.cuh"
#include "rk.cuh"

using namespace nm;

int fail(int code, const char *fmt, ...);
void clear_error();  // every entry point starts with this, so nm_last_error() describes its own failure

#define CUDA_TRY(expr)                                                                                     \
    do {                                                                                                   \
        cudaError_t _e = (expr);                                                                           \
        if (_e != cudaSuccess) return fail(NM_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e),   \
                                           __FILE__, __LINE__);                                            \
    } while (0)

#define CHECK_LAUNCH()                                                                                     \
    do {                                                                                                   \
        cudaError_t _e = cudaGetLastError();                                                               \
        if (_e != cudaSuccess) return fail(NM_ERR_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(_e), \
                                           __FILE__, __LINE__);                                            \
    } while (0)

// Dormand & Prince (1980) RK5(4)7M coefficients
static constexpr double kDpC[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static constexpr double kDpA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
static constexpr double kDpB[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
static constexpr double kDpBs[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100,
                                1.0 / 40};
// classical RK4
static constexpr double kRk4A[4][3] = {{0, 0, 0}, {0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 1.0}};
static constexpr double kRk4C[4] = {0.0, 0.5, 0.5, 1.0};
static constexpr double kRk4B[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};

struct nm_mesh_s {
    int prec;
    size_t rs;  // sizeof(real)
    cudaStream_t st;
    bool own_stream;
    Geom g;
    double dx[3];
    // device buffers
    double *m = nullptr;
    float *mf = nullptr;     // FP32 copy of m (FP32 meshes): kept equal to fl32(m) by the step updates
    bool mf_valid = false;   // false after m changed outside the step graphs
    void *y[2] = {nullptr, nullptr};
    void *k[7] = {};
    void *hin = nullptr, *hout = nullptr;
    void *inv_mass = nullptr, *vol = nullptr;
    void *MsH = nullptr;
    void *S = nullptr;
    void *Nk = nullptr;
    void *tw = nullptr;
    Cx<double> *tw64 = nullptr;
    void *A_d = nullptr, *Ku_d = nullptr, *Ms_d = nullptr;
    double *Ms64_d = nullptr;
    void *Msh_d = nullptr;
    void *D_d = nullptr;       // interfacial DMI per cell (working precision) or NULL: uniform D0
    void *hdmi = nullptr;      // raw DMI field -dE_DMI at the current stage input (3 x ns)
    double D0 = 0.0;
    bool has_dmi = false;
    double *hcell64_d = nullptr;
    StepCtl *ctl = nullptr;
    StepCtl *hctl = nullptr;  // pinned host mirror
    double *partials = nullptr;
    double *mean_d = nullptr;
    double *mean_h = nullptr;  // pinned
    unsigned long long *n_active_d = nullptr;
    // model
    double A0 = 0, Ku0 = 0, Ms0 = 0, axis[3] = {0, 0, 1}, alpha = 0, gamma = 0;
    double hu[3] = {0, 0, 0}, hu_freq = 0, hu_phase = 0, hc_freq = 0, hc_phase = 0;
    bool has_hcell = false;
    bool material_set = false, state_set = false, k1_valid = false;
    unsigned terms = NM_ALL;
    int renorm = 1;
    double dt_min = 1e-22;
    int max_rej = 50;
    double n_active = 0;
    long bytes = 0;
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
    // adjoint workspaces (allocated on first use)
    void *vj_w = nullptr, *vj_h = nullptr, *vj_q = nullptr, *vj_g = nullptr;      // nodal 3 x ns
    void *vj_H = nullptr, *vj_HW = nullptr, *vj_M = nullptr;                      // cells 3 x cs
    double *vj_gMs = nullptr;                                                    // cells, FP64 accumulator
    double *vj_gh = nullptr;  // nodal FP64 accumulator of the uniform-field gradient (during nm_adjoint_run)
    std::vector<void *> extra;                                                   // further adjoint buffers
    // per-launch profiling (nm_profile_step)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<const char *> prof_names;
    size_t prof_n = 0;
    unsigned long long *n_bad_d = nullptr;  // nodes with non-finite values met by nm_set_state (device)
    int err_f64_terms = 0;  // FP32 meshes: per-node error-norm terms in FP64 (nm_set_error_norm)
    CUtensorMap ymap;       // TMA descriptor of a y-pass tile over S (all P2 rows)
};


int dev_alloc(nm_mesh M, void **p, size_t bytes);
void *mapped_host(const void *p);  // device address of mapped page-locked host memory, or NULL
// nm_create_mesh; with tensor_src a mesh of the same shape, cell size and precision, the twiddles and
// the tensor spectrum are copied from it on the device instead of being rebuilt
int create_mesh(int n1, int n2, int n3, double dx1, double dx2, double dx3, int precision, void *cuda_stream,
                nm_mesh tensor_src, nm_mesh *out, int basis = 3);
long mesh_footprint(int n1, int n2, int n3, int precision);
int pull_ctl(nm_mesh M);
int push_ctl(nm_mesh M);
void free_graphs(nm_mesh M);
int check_step_args(nm_mesh M, int method, double rtol, double atol);
int launch_step(nm_mesh M, int method);  // one step attempt of the captured step graph
int ensure_mf(nm_mesh M);                // refresh the FP32 copy of m if m changed outside the steps
int ensure_k1(nm_mesh M, int method);    // FSAL slope at the resident state when not valid

// device buffer owned by the mesh (freed with it)
inline int alloc_extra(nm_mesh M, void **p, size_t bytes)
{
    int rc = dev_alloc(M, p, bytes);
    if (rc == NM_OK) M->extra.push_back(*p);
    return rc;
}

inline void prof_mark_cb(void *ctx, const char *name)
{
    nm_mesh M = (nm_mesh)ctx;
    if (!M->prof_on) return;
    if (M->prof_n == M->prof_ev.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        M->prof_ev.push_back(e);
        M->prof_names.push_back(name);
    }
    M->prof_names[M->prof_n] = name;
    cudaEventRecord(M->prof_ev[M->prof_n], M->st);
    ++M->prof_n;
}

inline Marker marker(nm_mesh M)
{
    Marker mk;
    if (M->prof_on) {
        mk.fn = prof_mark_cb;
        mk.ctx = M;
    }
    return mk;
}

template <typename T>
inline LocalParams<T> local_params(nm_mesh M, unsigned terms)
{
    LocalParams<T> p{};
    p.g = M->g;
    const double *dx = M->dx;
    const double V = dx[0] * dx[1] * dx[2];
    for (int d = 0; d < 8; ++d) {
        const int dd[3] = {(d >> 2) & 1, (d >> 1) & 1, d & 1};
        double kk = 0.0, mm = V;
        for (int k = 0; k < 3; ++k) mm *= dd[k] ? 1.0 / 6.0 : 1.0 / 3.0;
        for (int k = 0; k < 3; ++k) {
            double v = (dd[k] ? -1.0 : 1.0) / dx[k];
            for (int l = 0; l < 3; ++l)
                if (l != k) v *= dx[l] * (dd[l] ? 1.0 / 6.0 : 1.0 / 3.0);
            kk += v;
        }
        p.Wex[d] = (T)(2.0 * kk);
        p.Wm[d] = (T)mm;
    }
    p.mu0V8 = (T)(kMu0 * V / 8.0);
    p.mu0V4 = (T)(kMu0 * V / 4.0);
    for (int d = 0; d < 4; ++d) {
        const int d1 = (d >> 1) & 1, d2 = d & 1;
        const double M1x = dx[0] * (d1 ? 1.0 / 6.0 : 1.0 / 3.0), M1y = dx[1] * (d2 ? 1.0 / 6.0 : 1.0 / 3.0);
        const double K1x = (d1 ? -1.0 : 1.0) / dx[0], K1y = (d2 ? -1.0 : 1.0) / dx[1];
        p.Wex2[d] = (T)(2.0 * (K1x * M1y + M1x * K1y) * dx[2]);
        p.Wm2[d] = (T)(M1x * M1y * dx[2]);
    }
    p.mu0V2 = (T)(kMu0 * V / 2.0);
    for (int d = 0; d < 2; ++d) {
        const double M1x = dx[0] * (d ? 1.0 / 6.0 : 1.0 / 3.0), K1x = (d ? -1.0 : 1.0) / dx[0];
        p.Wex1[d] = (T)(2.0 * K1x * dx[1] * dx[2]);
        p.Wm1[d] = (T)(M1x * dx[1] * dx[2]);
    }
    p.A = (const T *)M->A_d;
    p.Ku = (const T *)M->Ku_d;
    p.Ms = (const T *)M->Ms_d;
    p.A0 = (T)M->A0;
    p.Ku0 = (T)M->Ku0;
    p.Ms0 = (T)M->Ms0;
    p.e0 = (T)M->axis[0]; p.e1 = (T)M->axis[1]; p.e2 = (T)M->axis[2];
    p.inv_mass = (const T *)M->inv_mass;
    p.MsH = (terms & NM_DEMAG) ? (const T *)M->MsH : nullptr;
    p.Msh = M->has_hcell ? (const T *)M->Msh_d : nullptr;
    p.hdmi = (M->has_dmi && (terms & NM_DMI) && M->g.basis == 3) ? (T *)M->hdmi : nullptr;
    p.Dm = (const T *)M->D_d;
    p.D0 = (T)M->D0;
    for (int d = 0; d < 4; ++d) {
        // DMI weights: int phi_i d_x phi_i' = o1 * (y, z mass integrals of the pattern), o1 = i1' - i1
        const int a = (d >> 1) & 1, b = d & 1;
        p.dmx[d] = (T)(dx[1] * (a ? 1.0 / 6.0 : 1.0 / 3.0) * dx[2] * (b ? 1.0 / 6.0 : 1.0 / 3.0));  // (|o2|, |o3|)
        p.dmy[d] = (T)(dx[0] * (a ? 1.0 / 6.0 : 1.0 / 3.0) * dx[2] * (b ? 1.0 / 6.0 : 1.0 / 3.0));  // (|o1|, |o3|)
    }
    p.hu0 = M->hu[0]; p.hu1 = M->hu[1]; p.hu2 = M->hu[2];
    p.hu_freq = M->hu_freq; p.hu_phase = M->hu_phase;
    p.hc_freq = M->hc_freq; p.hc_phase = M->hc_phase;
    p.terms = terms;
    // interior weights of a uniform material: each offset o couples through 2^(number of zero components)
    // cells, all with the same A and Ku
    p.uniform = (!M->Ms_d && !M->A_d && !M->Ku_d && M->Ms0 > 0.0) ? 1 : 0;
    {
        const double A = (terms & NM_EXCH) ? M->A0 : 0.0, Ku = (terms & NM_ANIS) ? M->Ku0 : 0.0;
        double wsum = 0.0;
        for (int o3 = -1; o3 <= 1; ++o3)
            for (int o2 = -1; o2 <= 1; ++o2)
                for (int o1 = -1; o1 <= 1; ++o1) {
                    const int d = ((o1 != 0) << 2) | ((o2 != 0) << 1) | (o3 != 0);
                    const int cnt = (o1 == 0 ? 2 : 1) * (o2 == 0 ? 2 : 1) * (o3 == 0 ? 2 : 1);
                    const int k = (o3 + 1) * 9 + (o2 + 1) * 3 + (o1 + 1);
                    const bool self = o1 == 0 && o2 == 0 && o3 == 0;
                    double wx = 0.0, wm = V;
                    for (int kk = 0; kk < 3; ++kk) {
                        const int dk = (d >> (2 - kk)) & 1;
                        double v = (dk ? -1.0 : 1.0) / dx[kk];
                        for (int l = 0; l < 3; ++l)
                            if (l != kk) v *= dx[l] * (((d >> (2 - l)) & 1) ? 1.0 / 6.0 : 1.0 / 3.0);
                        wx += v;
                        wm *= dk ? 1.0 / 6.0 : 1.0 / 3.0;
                    }
                    const double we = self ? 0.0 : 2.0 * wx * A * cnt;
                    p.wex27[k] = (T)we;
                    p.wan27[k] = (T)(wm * Ku * cnt);
                    wsum += we;
                }
        p.wex_sum = (T)wsum;
        for (int d = 0; d < 8; ++d) {
            p.wexd[d] = (T)((double)p.Wex[d] * A);
            p.wand[d] = (T)((double)p.Wm[d] * Ku);
        }
    }
    p.gam = M->gamma / (1.0 + M->alpha * M->alpha);
    p.alpha = M->alpha;
    p.gam_t = (T)p.gam;
    p.alpha_t = (T)p.alpha;
    return p;
}

template <typename T>
inline DemagBufs<T> demag_bufs(nm_mesh M)
{
    DemagBufs<T> b;
    b.S = (Cx<T> *)M->S;
    b.Nk = (const T *)M->Nk;
    b.tw = (const Cx<T> *)M->tw;
    b.Ms = (const T *)M->Ms_d;
    b.Ms0 = (T)M->Ms0;
    b.ctl = nullptr;
    b.mark = marker(M);
    b.ymap = &M->ymap;
    b.wait_err = &M->ctl->status;
    return b;
}

