// Transposed products used by the gradient of the effective field and by the discrete adjoint of the
// Runge-Kutta steps.
#include "vjp.cuh"

namespace nm {

template <typename T>
__global__ void k_scale_inv_mass(long n_nodes, long ns, const T *__restrict__ v, const T *__restrict__ im,
                                 T *__restrict__ w)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    const T s = im[n];
    for (int c = 0; c < 3; ++c) w[c * ns + n] = s > T(0) ? v[c * ns + n] * s : T(0);
}

template <typename T>
__global__ void k_cell_moment(Geom g, const T *__restrict__ y, const T *__restrict__ Ms, T Ms0, T scale,
                              T *__restrict__ out)
{
    long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (c >= g.n_cells) return;
    const int c1 = (int)(c % g.N1);
    const long r = c / g.N1;
    const int c2 = (int)(r % g.N2);
    const int c3 = (int)(r / g.N2);
    // corner offsets of the nodal basis: nn1 and nn1 nn2 for the trilinear basis; 0 along the directions
    // in which the 2D or 1D basis is constant, where the 8-corner sum counts each node twice (or 4 times)
    const long sy = g.ysn, sz = g.zsn;
    const long n0 = (long)c3 * sz + (long)c2 * sy + c1;
    const T ms = Ms ? Ms[c] : Ms0;
    for (int k = 0; k < 3; ++k) {
        const T *p = y + k * g.ns + n0;
        T s = (p[0] + p[1]) + (p[sy] + p[sy + 1]) + (p[sz] + p[sz + 1]) + (p[sz + sy] + p[sz + sy + 1]);
        out[k * g.cs + c] = ms * scale * s;
    }
}

template <typename T>
__global__ void k_grad_Ms(Geom g, GradMsArgs a, const T *__restrict__ im, double *__restrict__ gMs)
{
    long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (c >= g.n_cells) return;
    const int c1 = (int)(c % g.N1);
    const long r = c / g.N1;
    const int c2 = (int)(r % g.N2);
    const int c3 = (int)(r / g.N2);
    // corner offsets as in k_cell_moment: with the 2D and 1D bases the 8 corners collapse onto the
    // cell's 4 (2) nodes, which gives the gradient of the restricted system (basis functions that are
    // sums of trilinear ones, integrals V/4 or V/2 per cell)
    const long sy = g.ysn, sz = g.zsn;
    const long n0 = (long)c3 * sz + (long)c2 * sy + c1;
    const long off[8] = {0, 1, sy, sy + 1, sz, sz + 1, sz + sy, sz + sy + 1};
    const T *m = (const T *)a.m, *w = (const T *)a.w, *h = (const T *)a.h;
    double acc = 0.0;
    for (int k = 0; k < 3; ++k) {
        double W = 0.0, mb = 0.0, mass_term = 0.0;
        for (int i = 0; i < 8; ++i) {
            const long n = k * g.ns + n0 + off[i];
            const double wn = (double)w[n];
            W += wn;
            mb += (double)m[n];
            mass_term += wn * ((double)h[n] - a.hu[k]);
        }
        mb *= 0.125;
        double Hc = 0.0, HWc = 0.0;
        if (a.demag) {
            Hc = (double)((const T *)a.H)[k * g.cs + c];
            HWc = (double)((const T *)a.HW)[k * g.cs + c];
        }
        if (a.hcell) Hc += a.sc * a.hcell[k * g.cs + c];
        acc += W * Hc + mb * HWc - mass_term;
    }
    gMs[c] += a.weight * a.mu0V8 * acc;
}

template <typename T>
__global__ void k_llg_vjp_local(long n_nodes, long ns, const T *__restrict__ y, const T *__restrict__ H,
                                const T *__restrict__ u, const T *__restrict__ im, T gam, T alpha,
                                T *__restrict__ ybar, T *__restrict__ q)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    T yv[3], Hv[3], uv[3];
    for (int k = 0; k < 3; ++k) {
        yv[k] = y[k * ns + n];
        Hv[k] = H[k * ns + n];
        uv[k] = u[k * ns + n];
    }
    auto cross = [](const T *a, const T *b, T *c) {
        c[0] = a[1] * b[2] - a[2] * b[1];
        c[1] = a[2] * b[0] - a[0] * b[2];
        c[2] = a[0] * b[1] - a[1] * b[0];
    };
    T yb[3] = {0, 0, 0}, qv[3] = {0, 0, 0};
    if (im[n] > T(0)) {
        T Hxu[3], yxH[3], yxHxu[3], uxy[3], Hxuxy[3], uxyxy[3];
        cross(Hv, uv, Hxu);
        cross(yv, Hv, yxH);
        cross(yxH, uv, yxHxu);
        cross(uv, yv, uxy);
        cross(Hv, uxy, Hxuxy);
        cross(uxy, yv, uxyxy);
        for (int k = 0; k < 3; ++k) {
            yb[k] = -gam * (Hxu[k] + alpha * (yxHxu[k] + Hxuxy[k]));
            qv[k] = -gam * (uxy[k] + alpha * uxyxy[k]);
        }
    }
    for (int k = 0; k < 3; ++k) {
        ybar[k * ns + n] = yb[k];
        q[k * ns + n] = qv[k];
    }
}

template <typename T>
__global__ void k_axpby(long n_nodes, long ns, T a, const T *__restrict__ x, T b, const T *__restrict__ y,
                        T *__restrict__ out)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    for (int k = 0; k < 3; ++k) out[k * ns + n] = a * x[k * ns + n] + b * y[k * ns + n];
}

// ---------------------------------------------------------------------------------------------
template <typename T>
void launch_scale_inv_mass(const Geom &g, const T *v, const T *inv_mass, T *w, cudaStream_t st)
{
    k_scale_inv_mass<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g.n_nodes, g.ns, v, inv_mass, w);
}

template <typename T>
void launch_cell_moment(const Geom &g, const T *y, const T *Ms, T Ms0, T scale, T *out, cudaStream_t st)
{
    k_cell_moment<T><<<div_up(g.n_cells, 256), 256, 0, st>>>(g, y, Ms, Ms0, scale, out);
}

template <typename T>
void launch_grad_Ms(const Geom &g, const GradMsArgs &a, const T *inv_mass, double *gMs, cudaStream_t st)
{
    k_grad_Ms<T><<<div_up(g.n_cells, 256), 256, 0, st>>>(g, a, inv_mass, gMs);
}

template <typename T>
void launch_llg_vjp_local(const Geom &g, const T *y, const T *H, const T *u, const T *inv_mass, double gam,
                          double alpha, T *ybar, T *q, cudaStream_t st)
{
    k_llg_vjp_local<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g.n_nodes, g.ns, y, H, u, inv_mass, (T)gam, (T)alpha,
                                                                 ybar, q);
}

template <typename T>
void launch_axpby(const Geom &g, T a, const T *x, T b, const T *y, T *out, cudaStream_t st)
{
    k_axpby<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g.n_nodes, g.ns, a, x, b, y, out);
}

#define NM_VJP_INST(T)                                                                                          \
    template void launch_scale_inv_mass<T>(const Geom &, const T *, const T *, T *, cudaStream_t);               \
    template void launch_cell_moment<T>(const Geom &, const T *, const T *, T, T, T *, cudaStream_t);            \
    template void launch_grad_Ms<T>(const Geom &, const GradMsArgs &, const T *, double *, cudaStream_t);         \
    template void launch_llg_vjp_local<T>(const Geom &, const T *, const T *, const T *, const T *, double,      \
                                          double, T *, T *, cudaStream_t);                                      \
    template void launch_axpby<T>(const Geom &, T, const T *, T, const T *, T *, cudaStream_t);
NM_VJP_INST(float)
NM_VJP_INST(double)

}  // namespace nm

namespace nm {

// internal cell layout (c1 fastest, FP64) -> boundary layout (c1 slowest) in type To
template <typename To>
__global__ void k_cells_to_boundary(Geom g, const double *__restrict__ s, To *__restrict__ a)
{
    long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (c >= g.n_cells) return;
    const int c1 = (int)(c % g.N1);
    const long r = c / g.N1;
    const int c2 = (int)(r % g.N2);
    const int c3 = (int)(r / g.N2);
    a[((long)c1 * g.N2 + c2) * g.N3 + c3] = (To)s[c];
}

template <typename To>
void launch_cells_to_boundary(const Geom &g, const double *s, To *a, cudaStream_t st)
{
    k_cells_to_boundary<To><<<div_up(g.n_cells, 256), 256, 0, st>>>(g, s, a);
}
template void launch_cells_to_boundary<float>(const Geom &, const double *, float *, cudaStream_t);
template void launch_cells_to_boundary<double>(const Geom &, const double *, double *, cudaStream_t);

}  // namespace nm

namespace nm {

template <typename T>
__global__ void k_lincomb(long n_nodes, long ns, LinComb lc, T *__restrict__ out)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    for (int c = 0; c < 3; ++c) {
        const long i = c * ns + n;
        double acc = 0.0;
        for (int j = 0; j < lc.nt; ++j) acc += lc.at[j] * (double)((const T *)lc.pt[j])[i];
        for (int j = 0; j < lc.nd; ++j) acc += lc.ad[j] * lc.pd[j][i];
        out[i] = (T)acc;
    }
}

template <typename T>
__global__ void k_lincomb_d(long n_nodes, long ns, LinComb lc, double *__restrict__ out)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    for (int c = 0; c < 3; ++c) {
        const long i = c * ns + n;
        double acc = 0.0;
        for (int j = 0; j < lc.nt; ++j) acc += lc.at[j] * (double)((const T *)lc.pt[j])[i];
        for (int j = 0; j < lc.nd; ++j) acc += lc.ad[j] * lc.pd[j][i];
        out[i] = acc;
    }
}

template <typename T>
__global__ void k_renorm_adjoint(long n_nodes, long ns, const double *__restrict__ m, LinComb kb, double dt,
                                 const double *__restrict__ lam, int renorm, double *__restrict__ lam_t,
                                 T *__restrict__ lam_tw)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    double mt[3], l[3];
    for (int c = 0; c < 3; ++c) {
        const long i = c * ns + n;
        double acc = 0.0;
        for (int j = 0; j < kb.nt; ++j) acc += kb.at[j] * (double)((const T *)kb.pt[j])[i];
        mt[c] = m[i] + dt * acc;
        l[c] = lam[i];
    }
    if (renorm) {
        const double s = sqrt(mt[0] * mt[0] + mt[1] * mt[1] + mt[2] * mt[2]);
        if (s > 0.0) {
            const double h0 = mt[0] / s, h1 = mt[1] / s, h2 = mt[2] / s;
            const double d = h0 * l[0] + h1 * l[1] + h2 * l[2];
            l[0] = (l[0] - d * h0) / s;
            l[1] = (l[1] - d * h1) / s;
            l[2] = (l[2] - d * h2) / s;
        }
    }
    for (int c = 0; c < 3; ++c) {
        lam_t[c * ns + n] = l[c];
        lam_tw[c * ns + n] = (T)l[c];
    }
}

__global__ void __launch_bounds__(256) k_loss_terms(long n_nodes, long ns, const double *__restrict__ m,
                                                    const double *__restrict__ W, const double *__restrict__ tg,
                                                    double *__restrict__ lam, double *__restrict__ partials)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < n_nodes; n += (long)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) {
            const long i = c * ns + n;
            const double d = m[i] - (tg ? tg[i] : 0.0);
            acc += W[i] * d * d;
            if (lam) lam[i] += 2.0 * W[i] * d;
        }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(1024) k_sum_partials(const double *__restrict__ p, int n, double *out)
{
    __shared__ double sh[1024];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

template <typename T>
void launch_lincomb(const Geom &g, const LinComb &lc, T *out, cudaStream_t st)
{
    k_lincomb<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g.n_nodes, g.ns, lc, out);
}
template <typename T>
void launch_lincomb_d(const Geom &g, const LinComb &lc, double *out, cudaStream_t st)
{
    k_lincomb_d<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g.n_nodes, g.ns, lc, out);
}
template <typename T>
void launch_renorm_adjoint(const Geom &g, const double *m, const LinComb &kb, double dt, const double *lam,
                           int renorm, double *lam_t, T *lam_t_w, cudaStream_t st)
{
    k_renorm_adjoint<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g.n_nodes, g.ns, m, kb, dt, lam, renorm, lam_t,
                                                                  lam_t_w);
}
int launch_loss_terms(const Geom &g, const double *m, const double *W, const double *target, double *lam,
                      double *partials, cudaStream_t st)
{
    long b = (g.n_nodes + 255) / 256;
    int nb = (int)(b > 1024 ? 1024 : b);
    k_loss_terms<<<nb, 256, 0, st>>>(g.n_nodes, g.ns, m, W, target, lam, partials);
    return nb;
}
void launch_sum_partials(const double *partials, int n, double *out, cudaStream_t st)
{
    k_sum_partials<<<1, 1024, 0, st>>>(partials, n, out);
}

template <typename T>
__global__ void k_accum_nodal(long n_nodes, long ns, const T *__restrict__ q, double scale, double *__restrict__ acc)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    for (int c = 0; c < 3; ++c) acc[c * ns + n] += scale * (double)q[c * ns + n];
}

template <typename T>
void launch_accum_nodal(const Geom &g, const T *q, double scale, double *acc, cudaStream_t st)
{
    k_accum_nodal<T><<<(int)((g.n_nodes + 255) / 256), 256, 0, st>>>(g.n_nodes, g.ns, q, scale, acc);
}

__global__ void __launch_bounds__(256) k_sum_nodal3_partials(long n_nodes, long ns, const double *__restrict__ acc,
                                                              double *partials)
{
    __shared__ double sh[3][256];
    double v[3] = {0.0, 0.0, 0.0};
    for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < n_nodes; n += (long)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) v[c] += acc[c * ns + n];
    for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) partials[c * 1024 + blockIdx.x] = sh[c][0];
}

void launch_sum_nodal3(const Geom &g, const double *acc, double *partials, double *out, cudaStream_t st)
{
    long b = (g.n_nodes + 255) / 256;
    const int nb = (int)(b > 1024 ? 1024 : b);
    k_sum_nodal3_partials<<<nb, 256, 0, st>>>(g.n_nodes, g.ns, acc, partials);
    for (int c = 0; c < 3; ++c) k_sum_partials<<<1, 1024, 0, st>>>(partials + c * 1024, nb, out + c);
}

template void launch_accum_nodal<float>(const Geom &, const float *, double, double *, cudaStream_t);
template void launch_accum_nodal<double>(const Geom &, const double *, double, double *, cudaStream_t);

#define NM_ADJ_INST(T)                                                                                          \
    template void launch_lincomb<T>(const Geom &, const LinComb &, T *, cudaStream_t);                          \
    template void launch_lincomb_d<T>(const Geom &, const LinComb &, double *, cudaStream_t);                   \
    template void launch_renorm_adjoint<T>(const Geom &, const double *, const LinComb &, double, const double *, \
                                           int, double *, T *, cudaStream_t);
NM_ADJ_INST(float)
NM_ADJ_INST(double)

}  // namespace nm
