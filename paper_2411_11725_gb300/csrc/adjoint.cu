// Gradients: the transpose product of the effective field (nm_h_eff_vjp) and the discrete adjoint of
// the Runge-Kutta integration with checkpointed recomputation (nm_adjoint_run).
//
// The linear part of the effective field is h_lin(m) = -M^{-1} K m with K symmetric (exchange,
// anisotropy and demag derive from quadratic energies, Eqs. weak_form_discrete, mass_lumping), so
// J^T v = -K (v / mass): the forward node kernel evaluated on v / mass without the final division.
// The gradient with respect to the cell Ms map collects the three places Ms enters: the lumped mass,
// the Ms weights of the cell->node averages, and the demag source Ms_c m_c.
#include "mesh.cuh"
#include "vjp.cuh"

namespace {

template <typename T>
int ensure_vjp_buffers(nm_mesh M)
{
    const Geom &g = M->g;
    int rc;
    void **nod[] = {&M->vj_w, &M->vj_h, &M->vj_q, &M->vj_g};
    for (void **p : nod)
        if (!*p && (rc = dev_alloc(M, p, 3 * g.ns * sizeof(T)))) return rc;
    void **cel[] = {&M->vj_H, &M->vj_HW, &M->vj_M};
    for (void **p : cel)
        if (!*p && (rc = dev_alloc(M, p, 3 * g.cs * sizeof(T)))) return rc;
    if (!M->vj_gMs && (rc = dev_alloc(M, (void **)&M->vj_gMs, g.cs * sizeof(double)))) return rc;
    return NM_OK;
}

double host_time_factor(double f, double ph, double t)
{
    return f == 0.0 ? 1.0 : sin(2.0 * 3.14159265358979323846 * f * t + ph);
}

// h = h_eff(y) at time t for `terms` (full field, the forward kernels)
template <typename T>
void field_at(nm_mesh M, const T *y, unsigned terms, double t, T *h)
{
    if (terms & NM_DEMAG) demag_forward<T>(M->g, demag_bufs<T>(M), y, (T *)M->MsH, M->st);
    launch_heff<T>(local_params<T>(M, terms), y, h, t, M->st);
}

// gm = J_h(y)^T v (working precision); when gMs != NULL also gMs += weight * d<v, h(y)>/dMs using the
// forward field h (already evaluated at y and t).
template <typename T>
void heff_vjp_core(nm_mesh M, const T *y, const T *v, const T *h, unsigned terms, double t, T *gm, double *gMs,
                   double weight)
{
    const Geom &g = M->g;
    T *w = (T *)M->vj_w;
    launch_scale_inv_mass<T>(g, v, (const T *)M->inv_mass, w, M->st);
    LocalParams<T> pr = local_params<T>(M, terms & ~NM_ZEE);
    pr.raw = 1;
    if (terms & NM_DEMAG) demag_forward<T>(g, demag_bufs<T>(M), w, (T *)M->MsH, M->st);
    launch_heff<T>(pr, w, gm, t, M->st);
    if (!gMs) return;
    DemagBufs<T> b = demag_bufs<T>(M);
    const T *Ms = (const T *)M->Ms_d;
    if (terms & NM_DEMAG) {
        launch_cell_moment<T>(g, y, Ms, (T)M->Ms0, T(0.125), (T *)M->vj_M, M->st);
        demag_cells<T>(g, b, (const T *)M->vj_M, (T *)M->vj_H, M->st);
        launch_cell_moment<T>(g, w, Ms, (T)M->Ms0, T(1), (T *)M->vj_M, M->st);
        demag_cells<T>(g, b, (const T *)M->vj_M, (T *)M->vj_HW, M->st);
    }
    GradMsArgs a{};
    a.m = y;
    a.w = w;
    a.h = h;
    a.H = M->vj_H;
    a.HW = M->vj_HW;
    const bool zee = (terms & NM_ZEE) != 0;
    a.hcell = (zee && M->has_hcell) ? M->hcell64_d : nullptr;
    a.sc = host_time_factor(M->hc_freq, M->hc_phase, t);
    const double su = zee ? host_time_factor(M->hu_freq, M->hu_phase, t) : 0.0;
    for (int k = 0; k < 3; ++k) a.hu[k] = M->hu[k] * su;
    a.mu0V8 = kMu0 * M->dx[0] * M->dx[1] * M->dx[2] / 8.0;
    a.demag = (terms & NM_DEMAG) ? 1 : 0;
    a.weight = weight;
    launch_grad_Ms<T>(g, a, (const T *)M->inv_mass, gMs, M->st);
}

template <typename T>
int heff_vjp_t(nm_mesh M, const void *m, const void *v, unsigned terms, double t, void *grad_m, void *grad_Ms)
{
    int rc = ensure_vjp_buffers<T>(M);
    if (rc) return rc;
    const Geom &g = M->g;
    launch_aos_to_soa<T, T>(g, (const T *)m, (T *)M->hin, M->st);
    launch_aos_to_soa<T, T>(g, (const T *)v, (T *)M->vj_q, M->st);
    double *gMs = nullptr;
    if (grad_Ms) {
        CUDA_TRY(cudaMemsetAsync(M->vj_gMs, 0, g.cs * sizeof(double), M->st));
        field_at<T>(M, (const T *)M->hin, terms, t, (T *)M->vj_h);
        gMs = M->vj_gMs;
    }
    heff_vjp_core<T>(M, (const T *)M->hin, (const T *)M->vj_q, (const T *)M->vj_h, terms, t, (T *)M->vj_g, gMs, 1.0);
    launch_soa_to_aos<T, T>(g, (const T *)M->vj_g, (T *)grad_m, M->st);
    if (grad_Ms) launch_cells_to_boundary<T>(g, M->vj_gMs, (T *)grad_Ms, M->st);
    CHECK_LAUNCH();
    return NM_OK;
}

}  // namespace

extern "C" int nm_h_eff_vjp(nm_mesh M, const void *m, const void *v, unsigned terms, double t, void *grad_m,
                            void *grad_Ms)
{
    clear_error();
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (!m || !v || !grad_m) return fail(NM_ERR_ARG, "m, v and grad_m are required");
    if (terms & ~NM_TERMS_MASK) return fail(NM_ERR_ARG, "unknown term bits 0x%x", terms);
    if (!isfinite(t)) return fail(NM_ERR_ARG, "t must be finite");
    if (!M->material_set) return fail(NM_ERR_STATE, "material not set");
    return M->prec == NM_F64 ? heff_vjp_t<double>(M, m, v, terms, t, grad_m, grad_Ms)
                             : heff_vjp_t<float>(M, m, v, terms, t, grad_m, grad_Ms);
}

// ------------------------------------------------------------------------------------------------
// Discrete adjoint of the Runge-Kutta integration (backpropagation through the accepted steps with
// the step sizes of the forward run frozen).
//
// Step n maps (m_n, k1_n) to m_{n+1} = N(m_n + dt sum_j b_j k_j) (N: renormalisation, when on) and, for
// Dormand-Prince with FSAL, k1_{n+1} = k_7.  Going back with the adjoints (lam, mu) of (m_{n+1},
// k1_{n+1}):
//   lam~  = J_N^T lam
//   kbar_s = dt b_s lam~ + [s = 7] mu + sum_{i>s} dt a_is ybar_i,   ybar_s = J_f(y_s)^T kbar_s
//   mu_n  = kbar_1 (Dormand-Prince; RK4 takes ybar_1 = J_f(y_1)^T kbar_1 instead)
//   lam_n = lam~ + sum_s ybar_s
// and the Ms gradient gathers every (d f / d Ms)^T kbar_s.  Segments of `checkpoint_every` steps are
// recomputed from stored states, then walked backwards step by step.
namespace {

struct Tableau {
    int S;                // stages
    bool fsal;
    const double *c;
    double a[8][8];       // a[s][j], s, j 0-based
    double b[8];
};

Tableau tableau(int method)
{
    Tableau tb{};
    if (method == NM_DP54) {
        tb.S = 7;
        tb.fsal = true;
        tb.c = kDpC;
        for (int s = 0; s < 7; ++s) {
            for (int j = 0; j < 6; ++j) tb.a[s][j] = kDpA[s][j];
            tb.b[s] = kDpB[s];
        }
    } else {
        tb.S = 4;
        tb.fsal = false;
        tb.c = kRk4C;
        for (int s = 0; s < 4; ++s) {
            for (int j = 0; j < 3; ++j) tb.a[s][j] = kRk4A[s][j];
            tb.b[s] = kRk4B[s];
        }
    }
    return tb;
}

template <typename T>
struct AdjBufs {
    T *Y[8];      // stage inputs y_1..y_S
    T *YB[8];     // stage adjoints ybar_1..ybar_S
    T *kbar, *mu, *lamT;
    double *lam, *lamt, *partials, *scalar;
};

int set_ctl(nm_mesh M, double t, double dt)
{
    int rc = pull_ctl(M);
    if (rc) return rc;
    M->hctl->t = t;
    M->hctl->dt = dt;
    M->hctl->t_end = 0.0;
    M->hctl->done = 0;
    M->hctl->status = NM_OK;
    return push_ctl(M);
}

// Stage inputs and slopes of one step at the resident m (and FSAL k1), t and dt in ctl: y_s -> Y[s-1],
// k_s -> M->k[s-1].
template <typename T>
void run_stages(nm_mesh M, const Tableau &tb, AdjBufs<T> &A)
{
    const Geom &g = M->g;
    const LocalParams<T> p = local_params<T>(M, M->terms);
    KList in{};
    if (tb.fsal) {
        in.p[0] = M->k[0];
        in.a[0] = tb.a[1][0];
        in.n = 1;
        launch_stage_input<T>(g, M->m, in, M->ctl, A.Y[1], M->st);
    } else {
        launch_stage_input<T>(g, M->m, in, M->ctl, A.Y[0], M->st);
    }
    for (int s = tb.fsal ? 2 : 1; s <= tb.S; ++s) {
        const T *ys = A.Y[s - 1];
        if (p.terms & NM_DEMAG) {
            DemagBufs<T> b = demag_bufs<T>(M);
            b.ctl = M->ctl;
            demag_forward<T>(g, b, ys, (T *)M->MsH, M->st);
        }
        StageArgs sa{};
        sa.m = M->m;
        for (int j = 0; j < 7; ++j) sa.k[j] = M->k[j];
        const bool next = s < tb.S;
        for (int j = 0; next && j < s; ++j) {
            sa.a[j] = tb.a[s][j];
            sa.af[j] = (float)tb.a[s][j];
        }
        sa.s = s;
        sa.a_s = next ? tb.a[s][s - 1] : 0.0;
        sa.af_s = (float)sa.a_s;
        sa.c_s = tb.c[s - 1];
        sa.ctl = M->ctl;
        launch_llg_stage<T>(p, ys, (T *)M->k[s - 1], next ? A.Y[s] : nullptr, sa, M->st);
    }
}

KList b_list(nm_mesh M, const Tableau &tb, int nk)
{
    KList kb{};
    for (int j = 0; j < nk; ++j)
        if (tb.b[j] != 0.0) {
            kb.p[kb.n] = M->k[j];
            kb.a[kb.n] = tb.b[j];
            ++kb.n;
        }
    return kb;
}

// m <- N(m + dt sum b_j k_j) and k1 <- k_S (FSAL), dt and t from ctl
template <typename T>
int finish_step(nm_mesh M, const Tableau &tb)
{
    launch_rk4_update<T>(M->g, M->m, b_list(M, tb, tb.S), M->ctl, M->renorm, M->st);
    if (tb.fsal)
        CUDA_TRY(cudaMemcpyAsync(M->k[0], M->k[tb.S - 1], 3 * M->g.ns * sizeof(T), cudaMemcpyDeviceToDevice, M->st));
    return NM_OK;
}

// ybar = J_f(y)^T u at time t (LLG right-hand side), gMs += its Ms part
template <typename T>
void llg_vjp(nm_mesh M, const T *y, double t, const T *u, T *ybar)
{
    const Geom &g = M->g;
    field_at<T>(M, y, M->terms, t, (T *)M->vj_h);
    launch_llg_vjp_local<T>(g, y, (const T *)M->vj_h, u, (const T *)M->inv_mass,
                            M->gamma / (1.0 + M->alpha * M->alpha), M->alpha, ybar, (T *)M->vj_q, M->st);
    // the uniform applied field adds h s(t) to H at every magnetic node: dL/dh += s(t) sum_n q_n
    if (M->vj_gh && (M->terms & NM_ZEE))
        launch_accum_nodal<T>(g, (const T *)M->vj_q, host_time_factor(M->hu_freq, M->hu_phase, t), M->vj_gh, M->st);
    heff_vjp_core<T>(M, y, (const T *)M->vj_q, (const T *)M->vj_h, M->terms, t, (T *)M->vj_g, M->vj_gMs, 1.0);
    launch_axpby<T>(g, T(1), ybar, T(1), (const T *)M->vj_g, ybar, M->st);
}

// adjoint of one step whose stages (Y, k) are in place; m is the step's initial state
template <typename T>
void step_adjoint(nm_mesh M, const Tableau &tb, AdjBufs<T> &A, double t, double dt)
{
    const Geom &g = M->g;
    launch_renorm_adjoint<T>(g, M->m, [&] {
        LinComb kb{};
        KList l = b_list(M, tb, tb.S);
        for (int j = 0; j < l.n; ++j) { kb.pt[j] = l.p[j]; kb.at[j] = l.a[j]; }
        kb.nt = l.n;
        return kb;
    }(), dt, A.lam, M->renorm, A.lamt, A.lamT, M->st);
    const int s_lo = tb.fsal ? 2 : 1;
    for (int s = tb.S; s >= s_lo; --s) {
        LinComb lc{};
        lc.pt[lc.nt] = A.lamT;
        lc.at[lc.nt++] = dt * tb.b[s - 1];
        if (tb.fsal && s == tb.S) {
            lc.pt[lc.nt] = A.mu;
            lc.at[lc.nt++] = 1.0;
        }
        for (int i = s + 1; i <= tb.S; ++i)
            if (tb.a[i - 1][s - 1] != 0.0) {
                lc.pt[lc.nt] = A.YB[i - 1];
                lc.at[lc.nt++] = dt * tb.a[i - 1][s - 1];
            }
        launch_lincomb<T>(g, lc, A.kbar, M->st);
        llg_vjp<T>(M, A.Y[s - 1], t + tb.c[s - 1] * dt, A.kbar, A.YB[s - 1]);
    }
    if (tb.fsal) {
        LinComb lc{};
        lc.pt[lc.nt] = A.lamT;
        lc.at[lc.nt++] = dt * tb.b[0];
        for (int i = 2; i <= tb.S; ++i)
            if (tb.a[i - 1][0] != 0.0) {
                lc.pt[lc.nt] = A.YB[i - 1];
                lc.at[lc.nt++] = dt * tb.a[i - 1][0];
            }
        launch_lincomb<T>(g, lc, A.mu, M->st);
    }
    LinComb lc{};
    lc.pd[0] = A.lamt;
    lc.ad[0] = 1.0;
    lc.nd = 1;
    for (int s = s_lo; s <= tb.S; ++s) {
        lc.pt[lc.nt] = A.YB[s - 1];
        lc.at[lc.nt++] = 1.0;
    }
    launch_lincomb_d<T>(g, lc, A.lam, M->st);
}

}  // namespace

namespace {

// loss terms of one sample at the resident m: returns the sample's loss (synchronises); when lam is
// non-NULL also lam += dL/dm
template <typename T>
int sample_loss(nm_mesh M, const double *W, const double *tgt, double *lam, AdjBufs<T> &A, double *out)
{
    int nb = launch_loss_terms(M->g, M->m, W, tgt, lam, A.partials, M->st);
    launch_sum_partials(A.partials, nb, A.scalar, M->st);
    CHECK_LAUNCH();
    CUDA_TRY(cudaMemcpyAsync(M->mean_h, A.scalar, sizeof(double), cudaMemcpyDeviceToHost, M->st));
    CUDA_TRY(cudaStreamSynchronize(M->st));
    *out = M->mean_h[0];
    return NM_OK;
}

template <typename T>
int adjoint_run_t(nm_mesh M, int method, double t_end, double rtol, double atol, double dt0, double sample_dt,
                  const double *weight, const double *target, int include_initial, long C, double *loss_out,
                  double *grad_Ms, double *grad_m0, long *n_steps_out, double *grad_h)
{
    const Geom &g = M->g;
    const size_t nb3 = 3 * g.ns * sizeof(T), nd3 = 3 * g.ns * sizeof(double);
    int rc = ensure_vjp_buffers<T>(M);
    if (rc) return rc;
    const Tableau tb = tableau(method);
    // The forward steps and their recomputation in the reverse sweep must follow the same arithmetic,
    // and the reverse sweep restores m from checkpoints: stage inputs are formed from the FP64 m during
    // this call (no FP32 copy of m), and the step graphs are recaptured around it.
    struct MfOff {
        nm_mesh M;
        float *mf;
        explicit MfOff(nm_mesh m) : M(m), mf(m->mf)
        {
            M->mf = nullptr;
            free_graphs(M);
        }
        ~MfOff()
        {
            M->mf = mf;
            M->mf_valid = false;
            free_graphs(M);
        }
    } mf_off(M);
    // workspaces of this call (stream-ordered, freed at the end)
    std::vector<void *> owned;
    auto galloc = [&](void **p, size_t bytes) -> int {
        cudaError_t e = cudaMallocAsync(p, bytes, M->st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(NM_ERR_OOM, "adjoint workspace allocation failed (%zu bytes)", bytes);
        }
        owned.push_back(*p);
        return NM_OK;
    };
    auto release_all = [&]() {
        M->vj_gh = nullptr;
        for (void *p : owned) cudaFreeAsync(p, M->st);
        owned.clear();
    };
#define ADJ_TRY(x)                \
    do {                          \
        int _r = (x);             \
        if (_r) {                 \
            release_all();        \
            return _r;            \
        }                         \
    } while (0)
    AdjBufs<T> A{};
    for (int s = 0; s < tb.S; ++s) {
        ADJ_TRY(galloc((void **)&A.Y[s], nb3));
        ADJ_TRY(galloc((void **)&A.YB[s], nb3));
    }
    ADJ_TRY(galloc((void **)&A.kbar, nb3));
    ADJ_TRY(galloc((void **)&A.mu, nb3));
    ADJ_TRY(galloc((void **)&A.lamT, nb3));
    ADJ_TRY(galloc((void **)&A.lam, nd3));
    ADJ_TRY(galloc((void **)&A.lamt, nd3));
    ADJ_TRY(galloc((void **)&A.partials, 1024 * sizeof(double)));
    ADJ_TRY(galloc((void **)&A.scalar, sizeof(double)));
    if (grad_h) {
        double *gh = nullptr;
        ADJ_TRY(galloc((void **)&gh, nd3));
        CUDA_TRY(cudaMemsetAsync(gh, 0, nd3, M->st));
        M->vj_gh = gh;  // llg_vjp accumulates the uniform-field gradient here
    }
    double *W = nullptr, *tgt = nullptr, *tmp = nullptr;
    ADJ_TRY(galloc((void **)&W, nd3));
    // tmp stages the nodal inputs and outputs and the cell-wise Ms gradient: with the 2D and 1D bases a
    // mesh can have more cells than nodal values
    const size_t tmp_bytes = (g.n_nodes * 3 > g.n_cells ? g.n_nodes * 3 : g.n_cells) * sizeof(double);
    ADJ_TRY(galloc((void **)&tmp, tmp_bytes));
    CUDA_TRY(cudaMemcpyAsync(tmp, weight, g.n_nodes * 3 * sizeof(double), cudaMemcpyHostToDevice, M->st));
    CUDA_TRY(cudaMemsetAsync(W, 0, nd3, M->st));
    launch_aos_to_soa<double, double>(g, tmp, W, M->st);
    if (target) {
        ADJ_TRY(galloc((void **)&tgt, nd3));
        CUDA_TRY(cudaMemcpyAsync(tmp, target, g.n_nodes * 3 * sizeof(double), cudaMemcpyHostToDevice, M->st));
        CUDA_TRY(cudaMemsetAsync(tgt, 0, nd3, M->st));
        launch_aos_to_soa<double, double>(g, tmp, tgt, M->st);
    }
    CUDA_TRY(cudaMemsetAsync(M->vj_gMs, 0, g.cs * sizeof(double), M->st));

    // ---------------- forward: adaptive (or fixed) steps, clipped to the sample times, with a tape
    ADJ_TRY(pull_ctl(M));
    StepCtl *h = M->hctl;
    const double t0 = h->t;
    double dt = dt0 > 0 ? dt0 : h->dt;
    if (!(dt > 0) || t_end <= t0) {
        release_all();
        return fail(NM_ERR_ARG, "need t_end > t and a positive step");
    }
    M->k1_valid = false;
    ADJ_TRY(ensure_k1(M, method));  // k1_0 = f(m_0)
    std::vector<double> ts, dts;
    std::vector<char> sample_end;
    std::vector<double *> ck_m;
    std::vector<T *> ck_k;
    auto checkpoint = [&]() -> int {
        double *pm = nullptr;
        T *pk = nullptr;
        int r = galloc((void **)&pm, nd3);
        if (!r && tb.fsal) r = galloc((void **)&pk, nb3);
        if (r) return r;
        CUDA_TRY(cudaMemcpyAsync(pm, M->m, nd3, cudaMemcpyDeviceToDevice, M->st));
        if (tb.fsal) CUDA_TRY(cudaMemcpyAsync(pk, M->k[0], nb3, cudaMemcpyDeviceToDevice, M->st));
        ck_m.push_back(pm);
        ck_k.push_back(pk);
        return NM_OK;
    };
    double loss = 0.0, ls;
    if (include_initial) {
        ADJ_TRY(sample_loss<T>(M, W, tgt, nullptr, A, &ls));
        loss += ls;
    }
    ADJ_TRY(checkpoint());
    const double tiny = 1e-12 * fabs(t_end);
    long ks = 1;
    double t = t0;
    while (t < t_end - tiny) {
        double target_t = t_end;
        if (sample_dt > 0) {
            const double tsamp = t0 + ks * sample_dt;
            if (tsamp < target_t) target_t = tsamp;
        }
        while (true) {
            ADJ_TRY(pull_ctl(M));
            h->t = t;
            h->dt = method == NM_RK4 ? dt0 : dt;
            if (h->dt > target_t - t) h->dt = target_t - t;
            h->t_end = target_t;
            h->rtol = rtol;
            h->atol = atol;
            h->done = 0;
            h->status = NM_OK;
            h->dt_min = M->dt_min;
            ADJ_TRY(push_ctl(M));
            const double t_before = t;
            ADJ_TRY(launch_step(M, method));
            ADJ_TRY(pull_ctl(M));
            if (h->status != NM_OK) {
                release_all();
                return fail(h->status, "forward integration failed at t=%g", h->t);
            }
            if (h->accepted) {
                ts.push_back(t_before);
                dts.push_back(h->dt_used);
                sample_end.push_back(0);
                if ((long)ts.size() % C == 0) ADJ_TRY(checkpoint());
            }
            t = h->t;
            if (method == NM_DP54) dt = h->dt_prop > 0 ? h->dt_prop : h->dt;
            if (h->done || t >= target_t - tiny) break;
        }
        const bool is_sample = sample_dt <= 0 ? (t >= t_end - tiny)
                                              : fabs(t - (t0 + ks * sample_dt)) <= tiny + 1e-9 * sample_dt;
        if (is_sample) {
            ADJ_TRY(sample_loss<T>(M, W, tgt, nullptr, A, &ls));
            loss += ls;
            if (!sample_end.empty()) sample_end.back() = 1;
            ++ks;
        }
    }
    const long n = (long)ts.size();
    if (!grad_Ms && !grad_m0 && !grad_h) {
        // the loss alone: no reverse sweep; the resident state stays at the end of the run
        ADJ_TRY(set_ctl(M, t, dt));
        M->k1_valid = false;
        CUDA_TRY(cudaStreamSynchronize(M->st));
        release_all();
        CUDA_TRY(cudaStreamSynchronize(M->st));
        *loss_out = loss;
        if (n_steps_out) *n_steps_out = n;
        return NM_OK;
    }
    double *m_end = nullptr;
    ADJ_TRY(galloc((void **)&m_end, nd3));
    CUDA_TRY(cudaMemcpyAsync(m_end, M->m, nd3, cudaMemcpyDeviceToDevice, M->st));
    const double t_final = t, dt_final = dt;

    // ---------------- backward over the segments
    CUDA_TRY(cudaMemsetAsync(A.lam, 0, nd3, M->st));
    CUDA_TRY(cudaMemsetAsync(A.mu, 0, nb3, M->st));
    std::vector<double *> seg_m(C + 1, nullptr);
    std::vector<T *> seg_k(C + 1, nullptr);
    for (long i = 0; i <= C; ++i) {
        ADJ_TRY(galloc((void **)&seg_m[i], nd3));
        if (tb.fsal) ADJ_TRY(galloc((void **)&seg_k[i], nb3));
    }
    const long nseg = (n + C - 1) / C;
    for (long seg = nseg - 1; seg >= 0; --seg) {
        const long s0 = seg * C, s1 = (s0 + C < n) ? s0 + C : n;
        CUDA_TRY(cudaMemcpyAsync(M->m, ck_m[seg], nd3, cudaMemcpyDeviceToDevice, M->st));
        if (tb.fsal) CUDA_TRY(cudaMemcpyAsync(M->k[0], ck_k[seg], nb3, cudaMemcpyDeviceToDevice, M->st));
        for (long j = s0; j <= s1; ++j) {
            CUDA_TRY(cudaMemcpyAsync(seg_m[j - s0], M->m, nd3, cudaMemcpyDeviceToDevice, M->st));
            if (tb.fsal) CUDA_TRY(cudaMemcpyAsync(seg_k[j - s0], M->k[0], nb3, cudaMemcpyDeviceToDevice, M->st));
            if (j == s1) break;
            ADJ_TRY(set_ctl(M, ts[j], dts[j]));
            run_stages<T>(M, tb, A);
            ADJ_TRY(finish_step<T>(M, tb));
        }
        for (long j = s1 - 1; j >= s0; --j) {
            if (sample_end[j]) {
                CUDA_TRY(cudaMemcpyAsync(M->m, seg_m[j + 1 - s0], nd3, cudaMemcpyDeviceToDevice, M->st));
                ADJ_TRY(sample_loss<T>(M, W, tgt, A.lam, A, &ls));
            }
            CUDA_TRY(cudaMemcpyAsync(M->m, seg_m[j - s0], nd3, cudaMemcpyDeviceToDevice, M->st));
            if (tb.fsal) CUDA_TRY(cudaMemcpyAsync(M->k[0], seg_k[j - s0], nb3, cudaMemcpyDeviceToDevice, M->st));
            ADJ_TRY(set_ctl(M, ts[j], dts[j]));
            run_stages<T>(M, tb, A);
            step_adjoint<T>(M, tb, A, ts[j], dts[j]);
            CHECK_LAUNCH();
        }
    }
    // back at t0: the initial sample and, with FSAL, k1_0 = f(m_0)
    CUDA_TRY(cudaMemcpyAsync(M->m, ck_m[0], nd3, cudaMemcpyDeviceToDevice, M->st));
    if (include_initial) ADJ_TRY(sample_loss<T>(M, W, tgt, A.lam, A, &ls));
    if (tb.fsal) {
        KList none{};
        ADJ_TRY(set_ctl(M, t0, dt));
        launch_stage_input<T>(g, M->m, none, M->ctl, A.Y[0], M->st);
        llg_vjp<T>(M, A.Y[0], t0, A.mu, A.YB[0]);
        LinComb lc{};
        lc.pd[0] = A.lam;
        lc.ad[0] = 1.0;
        lc.nd = 1;
        lc.pt[0] = A.YB[0];
        lc.at[0] = 1.0;
        lc.nt = 1;
        launch_lincomb_d<T>(g, lc, A.lamt, M->st);
        CUDA_TRY(cudaMemcpyAsync(A.lam, A.lamt, nd3, cudaMemcpyDeviceToDevice, M->st));
    }
    CHECK_LAUNCH();
    // outputs
    if (grad_Ms) {
        launch_cells_to_boundary<double>(g, M->vj_gMs, tmp, M->st);
        CUDA_TRY(cudaMemcpyAsync(grad_Ms, tmp, g.n_cells * sizeof(double), cudaMemcpyDeviceToHost, M->st));
    }
    if (grad_m0) {
        launch_soa_to_aos<double, double>(g, A.lam, tmp, M->st);
        CUDA_TRY(cudaMemcpyAsync(grad_m0, tmp, g.n_nodes * 3 * sizeof(double), cudaMemcpyDeviceToHost, M->st));
    }
    if (grad_h) {
        launch_sum_nodal3(g, M->vj_gh, M->partials, M->mean_d, M->st);
        CHECK_LAUNCH();
        CUDA_TRY(cudaMemcpyAsync(M->mean_h, M->mean_d, 3 * sizeof(double), cudaMemcpyDeviceToHost, M->st));
        CUDA_TRY(cudaStreamSynchronize(M->st));
        for (int c = 0; c < 3; ++c) grad_h[c] = M->mean_h[c];
    }
    // leave the resident state at the end of the forward run (k1 recomputed on the next step)
    CUDA_TRY(cudaMemcpyAsync(M->m, m_end, nd3, cudaMemcpyDeviceToDevice, M->st));
    ADJ_TRY(set_ctl(M, t_final, dt_final));
    M->k1_valid = false;
    CHECK_LAUNCH();
    CUDA_TRY(cudaStreamSynchronize(M->st));
    release_all();
    CUDA_TRY(cudaStreamSynchronize(M->st));
    *loss_out = loss;
    if (n_steps_out) *n_steps_out = n;
    return NM_OK;
#undef ADJ_TRY
}

}  // namespace

extern "C" int nm_adjoint_run(nm_mesh M, int method, double t_end, double rtol, double atol, double dt0,
                              double sample_dt, const double *weight, const double *target, int include_initial,
                              long checkpoint_every, double *loss, double *grad_Ms, double *grad_m0, long *n_steps,
                              double *grad_h)
{
    clear_error();
    int rc = check_step_args(M, method, rtol, atol);
    if (rc) return rc;
    if (!weight || !loss) return fail(NM_ERR_ARG, "weight and loss are required");
    if (!isfinite(t_end) || !isfinite(dt0) || !isfinite(sample_dt)) return fail(NM_ERR_ARG, "non-finite argument");
    if (method == NM_RK4 && !(dt0 > 0)) return fail(NM_ERR_ARG, "RK4 needs dt0 > 0");
    if (checkpoint_every < 1) checkpoint_every = 32;
    return M->prec == NM_F64
               ? adjoint_run_t<double>(M, method, t_end, rtol, atol, dt0, sample_dt, weight, target, include_initial,
                                       checkpoint_every, loss, grad_Ms, grad_m0, n_steps, grad_h)
               : adjoint_run_t<float>(M, method, t_end, rtol, atol, dt0, sample_dt, weight, target, include_initial,
                                      checkpoint_every, loss, grad_Ms, grad_m0, n_steps, grad_h);
}

// ------------------------------------------------------------------------------------------------
// Continuous adjoint-state method (section "Inverse Micromagnetics", Eq. adjoint_system).
//
// The forward problem is integrated with n classical Runge-Kutta steps from the resident state to T.
// The system
//   dm/dt = f(t, m),   da/dt = -(df/dm)^T a,   du/dt = -(df/dtheta)^T a,
//   m(T) = m_output,   a(T) = dL/dm(T),        u(T) = 0
// is then integrated backwards with n steps of -dt.  The m stages are the forward stage kernels run
// with the negative step; they do not depend on a, so each step forms them first and then the a stages:
//   a_s = a + h sum_j A_sj ka_j,   ka_s = -(df/dm)(y_s)^T a_s,
// where the transpose product is evaluated on w_s a_s (w_s = -h b_s) so that the Ms and uniform-field
// accumulators of llg_vjp collect u's increments -h b_s (df/dtheta)^T a_s directly.  m is renormalised
// after each backward step when the forward steps renormalise.  Unlike the discrete adjoint, m is
// reconstructed by the backward integration, not read from checkpoints.
namespace {

template <typename T>
int continuous_adjoint_t(nm_mesh M, double t_end, long n, const double *weight, const double *target,
                         double *loss_out, double *grad_m0, double *grad_Ms, double *grad_h, double *m0_rec)
{
    const Geom &g = M->g;
    const size_t nb3 = 3 * g.ns * sizeof(T), nd3 = 3 * g.ns * sizeof(double);
    int rc = ensure_vjp_buffers<T>(M);
    if (rc) return rc;
    const Tableau tb = tableau(NM_RK4);
    struct MfOff {
        nm_mesh M;
        float *mf;
        explicit MfOff(nm_mesh m) : M(m), mf(m->mf)
        {
            M->mf = nullptr;
            free_graphs(M);
        }
        ~MfOff()
        {
            M->mf = mf;
            M->mf_valid = false;
            free_graphs(M);
        }
    } mf_off(M);
    std::vector<void *> owned;
    auto galloc = [&](void **p, size_t bytes) -> int {
        cudaError_t e = cudaMallocAsync(p, bytes, M->st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(NM_ERR_OOM, "adjoint workspace allocation failed (%zu bytes)", bytes);
        }
        owned.push_back(*p);
        return NM_OK;
    };
    auto release_all = [&]() {
        M->vj_gh = nullptr;
        for (void *p : owned) cudaFreeAsync(p, M->st);
        owned.clear();
    };
#define CA_TRY(x)                 \
    do {                          \
        int _r = (x);             \
        if (_r) {                 \
            release_all();        \
            return _r;            \
        }                         \
    } while (0)
    AdjBufs<T> A{};
    for (int s = 0; s < tb.S; ++s) {
        CA_TRY(galloc((void **)&A.Y[s], nb3));
        CA_TRY(galloc((void **)&A.YB[s], nb3));  // ka_s
    }
    T *C = nullptr, *YB = nullptr;
    double *a = nullptr, *as = nullptr, *W = nullptr, *tgt = nullptr, *tmp = nullptr, *m_end = nullptr;
    CA_TRY(galloc((void **)&C, nb3));
    CA_TRY(galloc((void **)&YB, nb3));
    CA_TRY(galloc((void **)&a, nd3));
    CA_TRY(galloc((void **)&as, nd3));
    CA_TRY(galloc((void **)&m_end, nd3));
    CA_TRY(galloc((void **)&A.partials, 1024 * sizeof(double)));
    CA_TRY(galloc((void **)&A.scalar, sizeof(double)));
    CA_TRY(galloc((void **)&W, nd3));
    const size_t tmp_bytes = (g.n_nodes * 3 > g.n_cells ? g.n_nodes * 3 : g.n_cells) * sizeof(double);
    CA_TRY(galloc((void **)&tmp, tmp_bytes));
    CUDA_TRY(cudaMemcpyAsync(tmp, weight, g.n_nodes * 3 * sizeof(double), cudaMemcpyHostToDevice, M->st));
    CUDA_TRY(cudaMemsetAsync(W, 0, nd3, M->st));
    launch_aos_to_soa<double, double>(g, tmp, W, M->st);
    if (target) {
        CA_TRY(galloc((void **)&tgt, nd3));
        CUDA_TRY(cudaMemcpyAsync(tmp, target, g.n_nodes * 3 * sizeof(double), cudaMemcpyHostToDevice, M->st));
        CUDA_TRY(cudaMemsetAsync(tgt, 0, nd3, M->st));
        launch_aos_to_soa<double, double>(g, tmp, tgt, M->st);
    }
    if (grad_h) {
        double *gh = nullptr;
        CA_TRY(galloc((void **)&gh, nd3));
        CUDA_TRY(cudaMemsetAsync(gh, 0, nd3, M->st));
        M->vj_gh = gh;
    }
    CUDA_TRY(cudaMemsetAsync(M->vj_gMs, 0, g.cs * sizeof(double), M->st));

    // forward: n RK4 steps to t_end
    CA_TRY(pull_ctl(M));
    const double t0 = M->hctl->t, dt = (t_end - t0) / (double)n;
    if (!(dt > 0)) {
        release_all();
        return fail(NM_ERR_ARG, "need t_end > t");
    }
    for (long k = 0; k < n; ++k) {
        CA_TRY(set_ctl(M, t0 + k * dt, dt));
        run_stages<T>(M, tb, A);
        CA_TRY(finish_step<T>(M, tb));
        CHECK_LAUNCH();
    }
    // loss and a(T) = dL/dm(T)
    CUDA_TRY(cudaMemsetAsync(a, 0, nd3, M->st));
    CA_TRY(sample_loss<T>(M, W, tgt, a, A, loss_out));
    CUDA_TRY(cudaMemcpyAsync(m_end, M->m, nd3, cudaMemcpyDeviceToDevice, M->st));

    // backward: n steps of -dt for (m, a, u)
    const double hb = -dt;
    for (long k = 0; k < n; ++k) {
        const double t = t_end - k * dt;
        CA_TRY(set_ctl(M, t, hb));
        run_stages<T>(M, tb, A);  // y_s in A.Y, f(y_s) in M->k
        for (int s = 1; s <= tb.S; ++s) {
            LinComb lc{};
            lc.pd[0] = a;
            lc.ad[0] = 1.0;
            lc.nd = 1;
            for (int j = 1; j < s; ++j)
                if (tb.a[s - 1][j - 1] != 0.0) {
                    lc.pt[lc.nt] = A.YB[j - 1];
                    lc.at[lc.nt++] = hb * tb.a[s - 1][j - 1];
                }
            launch_lincomb_d<T>(g, lc, as, M->st);
            const double w = -hb * tb.b[s - 1];
            LinComb sc{};
            sc.pd[0] = as;
            sc.ad[0] = w;
            sc.nd = 1;
            launch_lincomb<T>(g, sc, C, M->st);
            llg_vjp<T>(M, A.Y[s - 1], t + tb.c[s - 1] * hb, C, YB);
            launch_axpby<T>(g, T(-1.0 / w), YB, T(0), YB, A.YB[s - 1], M->st);
        }
        CA_TRY(finish_step<T>(M, tb));  // m <- N(m + h sum b_s f(y_s))
        LinComb lc{};
        lc.pd[0] = a;
        lc.ad[0] = 1.0;
        lc.nd = 1;
        for (int s = 1; s <= tb.S; ++s) {
            lc.pt[lc.nt] = A.YB[s - 1];
            lc.at[lc.nt++] = hb * tb.b[s - 1];
        }
        launch_lincomb_d<T>(g, lc, as, M->st);
        CUDA_TRY(cudaMemcpyAsync(a, as, nd3, cudaMemcpyDeviceToDevice, M->st));
        CHECK_LAUNCH();
    }
    // outputs
    if (grad_m0) {
        launch_soa_to_aos<double, double>(g, a, tmp, M->st);
        CUDA_TRY(cudaMemcpyAsync(grad_m0, tmp, g.n_nodes * 3 * sizeof(double), cudaMemcpyDeviceToHost, M->st));
        CUDA_TRY(cudaStreamSynchronize(M->st));
    }
    if (m0_rec) {
        launch_soa_to_aos<double, double>(g, M->m, tmp, M->st);
        CUDA_TRY(cudaMemcpyAsync(m0_rec, tmp, g.n_nodes * 3 * sizeof(double), cudaMemcpyDeviceToHost, M->st));
        CUDA_TRY(cudaStreamSynchronize(M->st));
    }
    if (grad_Ms) {
        launch_cells_to_boundary<double>(g, M->vj_gMs, tmp, M->st);
        CUDA_TRY(cudaMemcpyAsync(grad_Ms, tmp, g.n_cells * sizeof(double), cudaMemcpyDeviceToHost, M->st));
        CUDA_TRY(cudaStreamSynchronize(M->st));
    }
    if (grad_h) {
        launch_sum_nodal3(g, M->vj_gh, M->partials, M->mean_d, M->st);
        CHECK_LAUNCH();
        CUDA_TRY(cudaMemcpyAsync(M->mean_h, M->mean_d, 3 * sizeof(double), cudaMemcpyDeviceToHost, M->st));
        CUDA_TRY(cudaStreamSynchronize(M->st));
        for (int c = 0; c < 3; ++c) grad_h[c] = M->mean_h[c];
    }
    // leave the resident state at the end of the forward run
    CUDA_TRY(cudaMemcpyAsync(M->m, m_end, nd3, cudaMemcpyDeviceToDevice, M->st));
    CA_TRY(set_ctl(M, t_end, dt));
    M->k1_valid = false;
    CHECK_LAUNCH();
    CUDA_TRY(cudaStreamSynchronize(M->st));
    release_all();
    CUDA_TRY(cudaStreamSynchronize(M->st));
    return NM_OK;
#undef CA_TRY
}

}  // namespace

extern "C" int nm_adjoint_continuous(nm_mesh M, double t_end, long n_steps, const double *weight,
                                     const double *target, double *loss, double *grad_m0, double *grad_Ms,
                                     double *grad_h, double *m0_rec)
{
    clear_error();
    if (!M) return fail(NM_ERR_ARG, "mesh is NULL");
    if (!M->material_set) return fail(NM_ERR_STATE, "material not set");
    if (!M->state_set) return fail(NM_ERR_STATE, "no resident state");
    if (!weight || !loss) return fail(NM_ERR_ARG, "weight and loss are required");
    if (!isfinite(t_end)) return fail(NM_ERR_ARG, "non-finite argument");
    if (n_steps < 1) return fail(NM_ERR_ARG, "n_steps must be >= 1");
    return M->prec == NM_F64 ? continuous_adjoint_t<double>(M, t_end, n_steps, weight, target, loss, grad_m0, grad_Ms,
                                                            grad_h, m0_rec)
                             : continuous_adjoint_t<float>(M, t_end, n_steps, weight, target, loss, grad_m0, grad_Ms,
                                                           grad_h, m0_rec);
}
