// Fused node kernel: exchange, uniaxial anisotropy, Zeeman and the cell->node demag average, divided
// by the lumped nodal mass (Eqs. weak_form_impl_f, weak_form_impl, mass_lumping), followed by the LLG
// right-hand side (Eq. llg) and the formation of the next Runge-Kutta stage input.
//
// Assembly by neighbour instead of by cell: node n couples to n + o (o in {-1,0,1}^3) through every
// cell that holds both nodes; those are the cells c = n - i with i_k = 1 where o_k = -1, i_k = 0
// where o_k = +1 and either where o_k = 0.  The element integral of such a pair depends only on the
// pattern d = |o|, so the variation at n is
//   dE_ex,n = sum_o Wex[d(o)] (sum_{cells} A_c) (m_{n+o} - m_n)         (rows of Kex sum to zero)
//   dE_an,n = -2 e sum_o Wm[d(o)] (sum_{cells} Ku_c) (e . m_{n+o})
// which is the cell-by-cell sum of the paper regrouped per neighbour (a gather, no atomics).
#include "local.cuh"

namespace nm {

template <typename T>
__device__ __forceinline__ double time_factor(double f, double ph, double t)
{
    return f == 0.0 ? 1.0 : sin(2.0 * 3.14159265358979323846 * f * t + ph);
}

template <typename T>
struct NodeField {
    T hx, hy, hz;
    T mx, my, mz;
    bool magnetic;
};

// Applied-field factors at time t, computed once per block: (h_uniform * s_u(t), s_c(t)).
template <typename T>
__device__ __forceinline__ void block_field_factors(const LocalParams<T> &p, double t, T out[4])
{
    __shared__ T sh[4];
    if (threadIdx.x == 0) {
        const double su = time_factor<T>(p.hu_freq, p.hu_phase, t);
        sh[0] = (T)(p.hu0 * su);
        sh[1] = (T)(p.hu1 * su);
        sh[2] = (T)(p.hu2 * su);
        sh[3] = (T)time_factor<T>(p.hc_freq, p.hc_phase, t);
    }
    __syncthreads();
    out[0] = sh[0]; out[1] = sh[1]; out[2] = sh[2]; out[3] = sh[3];
}

template <typename T>
__device__ __forceinline__ NodeField<T> node_field(const LocalParams<T> &p, const T *__restrict__ y, long n,
                                                   const T hf[4])
{
    const Geom &g = p.g;
    const int n1 = (int)(n % g.nn1);
    const long r = n / g.nn1;
    const int n2 = (int)(r % g.nn2);
    const int n3 = (int)(r / g.nn2);
    T a[8], ku[8];
    long cidx[8];
    bool cval[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int c1 = n1 - ((i >> 2) & 1), c2 = n2 - ((i >> 1) & 1), c3 = n3 - (i & 1);
        bool valid = c1 >= 0 && c1 < g.N1 && c2 >= 0 && c2 < g.N2 && c3 >= 0 && c3 < g.N3;
        long c = valid ? ((long)c3 * g.N2 + c2) * g.N1 + c1 : 0;
        T Ms = valid ? (p.Ms ? p.Ms[c] : p.Ms0) : T(0);
        bool mag = valid && Ms > T(0);
        a[i] = (mag && (p.terms & NM_EXCH)) ? (p.A ? p.A[c] : p.A0) : T(0);
        ku[i] = (mag && (p.terms & NM_ANIS)) ? (p.Ku ? p.Ku[c] : p.Ku0) : T(0);
        cidx[i] = c;
        cval[i] = valid;
    }
    const long ns = g.ns;
    NodeField<T> f;
    f.mx = y[n];
    f.my = y[ns + n];
    f.mz = y[2 * ns + n];
    const T im = p.inv_mass[n];
    f.magnetic = im > T(0);
    T ex = 0, ey = 0, ez = 0, pe = 0;
    const long sy = g.nn1, sz = (long)g.nn1 * g.nn2;
#pragma unroll
    for (int o1 = -1; o1 <= 1; ++o1)
#pragma unroll
        for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
            for (int o3 = -1; o3 <= 1; ++o3) {
                T S = 0, K = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    int i1 = (i >> 2) & 1, i2 = (i >> 1) & 1, i3 = i & 1;
                    bool comp = (o1 == -1 ? i1 == 1 : (o1 == 1 ? i1 == 0 : true)) &&
                                (o2 == -1 ? i2 == 1 : (o2 == 1 ? i2 == 0 : true)) &&
                                (o3 == -1 ? i3 == 1 : (o3 == 1 ? i3 == 0 : true));
                    if (comp) { S += a[i]; K += ku[i]; }
                }
                const int d = ((o1 != 0) << 2) | ((o2 != 0) << 1) | (o3 != 0);
                const bool self = (o1 == 0 && o2 == 0 && o3 == 0);
                if ((!self && S != T(0)) || K != T(0)) {
                    long nb = n + o1 + o2 * sy + o3 * sz;
                    T qx = self ? f.mx : y[nb], qy = self ? f.my : y[ns + nb], qz = self ? f.mz : y[2 * ns + nb];
                    if (!self) {
                        T w = p.Wex[d] * S;
                        ex += w * (qx - f.mx);
                        ey += w * (qy - f.my);
                        ez += w * (qz - f.mz);
                    }
                    pe += p.Wm[d] * K * (p.e0 * qx + p.e1 * qy + p.e2 * qz);
                }
            }
    // -dE / mass: exchange and anisotropy
    T hx = -ex + T(2) * p.e0 * pe;
    T hy = -ey + T(2) * p.e1 * pe;
    T hz = -ez + T(2) * p.e2 * pe;
    // cell -> node: demag (Ms_c H_c) and cell applied field (Ms_c h_c), weight mu0 V/8
    T cx_ = 0, cy_ = 0, cz_ = 0;
    if (p.MsH && (p.terms & NM_DEMAG)) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (cval[i]) {
                cx_ += p.MsH[cidx[i]];
                cy_ += p.MsH[g.cs + cidx[i]];
                cz_ += p.MsH[2 * g.cs + cidx[i]];
            }
    }
    if (p.Msh && (p.terms & NM_ZEE)) {
        const T sc = hf[3];
        T ax = 0, ay = 0, az = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (cval[i]) {
                ax += p.Msh[cidx[i]];
                ay += p.Msh[g.cs + cidx[i]];
                az += p.Msh[2 * g.cs + cidx[i]];
            }
        cx_ += sc * ax;
        cy_ += sc * ay;
        cz_ += sc * az;
    }
    if (p.raw) {
        // -dE itself (the transpose products of the adjoint): no lumped-mass division
        f.hx = hx + p.mu0V8 * cx_;
        f.hy = hy + p.mu0V8 * cy_;
        f.hz = hz + p.mu0V8 * cz_;
        return f;
    }
    hx = im * (hx + p.mu0V8 * cx_);
    hy = im * (hy + p.mu0V8 * cy_);
    hz = im * (hz + p.mu0V8 * cz_);
    if (f.magnetic && (p.terms & NM_ZEE)) {
        hx += hf[0];
        hy += hf[1];
        hz += hf[2];
    }
    f.hx = hx; f.hy = hy; f.hz = hz;
    return f;
}

template <typename T>
__global__ void __launch_bounds__(256) k_heff(LocalParams<T> p, const T *__restrict__ y, T *__restrict__ h, double t)
{
    T hf[4];
    block_field_factors(p, t, hf);
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= p.g.n_nodes) return;
    NodeField<T> f = node_field(p, y, n, hf);
    const long ns = p.g.ns;
    h[n] = f.hx;
    h[ns + n] = f.hy;
    h[2 * ns + n] = f.hz;
}

template <typename T>
__global__ void __launch_bounds__(256) k_llg_stage(LocalParams<T> p, const T *__restrict__ y, T *__restrict__ k_out,
                                                   T *__restrict__ y_next, StageArgs sa)
{
    if (sa.ctl && sa.ctl->done) return;
    const double t = sa.ctl ? sa.ctl->t + sa.c_s * sa.ctl->dt : sa.t_fixed;
    T hf[4];
    block_field_factors(p, t, hf);
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= p.g.n_nodes) return;
    NodeField<T> f = node_field(p, y, n, hf);
    const long ns = p.g.ns;
    T kx = 0, ky = 0, kz = 0;
    if (f.magnetic) {
        // k = -gamma'(m x H + alpha m x (m x H))
        T ax = f.my * f.hz - f.mz * f.hy;
        T ay = f.mz * f.hx - f.mx * f.hz;
        T az = f.mx * f.hy - f.my * f.hx;
        T bx = f.my * az - f.mz * ay;
        T by = f.mz * ax - f.mx * az;
        T bz = f.mx * ay - f.my * ax;
        T gm = (T)p.gam, al = (T)p.alpha;
        kx = -gm * (ax + al * bx);
        ky = -gm * (ay + al * by);
        kz = -gm * (az + al * bz);
    }
    k_out[n] = kx;
    k_out[ns + n] = ky;
    k_out[2 * ns + n] = kz;
    if (y_next) {
        // y_{s+1} = m + dt sum_{j<=s} a_{s+1,j} k_j: the slope combination in the working precision,
        // the addition to the FP64 magnetisation in FP64
        const double dt = sa.ctl ? sa.ctl->dt : 0.0;
        T ax = 0, ay = 0, az = 0;
        for (int j = 0; j + 1 < sa.s; ++j) {
            const T aj = sizeof(T) == 4 ? (T)sa.af[j] : (T)sa.a[j];
            if (aj == T(0)) continue;
            const T *kj = (const T *)sa.k[j];
            ax += aj * kj[n];
            ay += aj * kj[ns + n];
            az += aj * kj[2 * ns + n];
        }
        const T as = sizeof(T) == 4 ? (T)sa.af[sa.s - 1] : (T)sa.a[sa.s - 1];
        ax += as * kx;
        ay += as * ky;
        az += as * kz;
        y_next[n] = (T)(sa.m[n] + dt * (double)ax);
        y_next[ns + n] = (T)(sa.m[ns + n] + dt * (double)ay);
        y_next[2 * ns + n] = (T)(sa.m[2 * ns + n] + dt * (double)az);
    }
}

template <typename T>
void launch_heff(const LocalParams<T> &p, const T *y, T *h_out, double t, cudaStream_t st)
{
    k_heff<T><<<div_up(p.g.n_nodes, 256), 256, 0, st>>>(p, y, h_out, t);
}

template <typename T>
void launch_llg_stage(const LocalParams<T> &p, const T *y, T *k_out, T *y_next, const StageArgs &sa, cudaStream_t st)
{
    k_llg_stage<T><<<div_up(p.g.n_nodes, 256), 256, 0, st>>>(p, y, k_out, y_next, sa);
}

// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_mass(Geom g, const double *__restrict__ Ms, double Ms0, double mu0V8, T *inv_mass,
                       unsigned long long *n_active)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= g.n_nodes) return;
    const int n1 = (int)(n % g.nn1);
    const long r = n / g.nn1;
    const int n2 = (int)(r % g.nn2);
    const int n3 = (int)(r / g.nn2);
    double s = 0.0;
    for (int i = 0; i < 8; ++i) {
        int c1 = n1 - ((i >> 2) & 1), c2 = n2 - ((i >> 1) & 1), c3 = n3 - (i & 1);
        if (c1 >= 0 && c1 < g.N1 && c2 >= 0 && c2 < g.N2 && c3 >= 0 && c3 < g.N3)
            s += Ms ? Ms[((long)c3 * g.N2 + c2) * g.N1 + c1] : Ms0;
    }
    double mass = mu0V8 * s;
    inv_mass[n] = mass > 0.0 ? (T)(1.0 / mass) : T(0);
    if (mass > 0.0) atomicAdd(n_active, 1ull);
}

template <typename T>
void launch_mass(const Geom &g, const double *Ms_d, double Ms0, double V, T *inv_mass, unsigned long long *n_active,
                 cudaStream_t st)
{
    k_mass<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g, Ms_d, Ms0, kMu0 * V / 8.0, inv_mass, n_active);
}

template void launch_heff<float>(const LocalParams<float> &, const float *, float *, double, cudaStream_t);
template void launch_heff<double>(const LocalParams<double> &, const double *, double *, double, cudaStream_t);
template void launch_llg_stage<float>(const LocalParams<float> &, const float *, float *, float *, const StageArgs &,
                                      cudaStream_t);
template void launch_llg_stage<double>(const LocalParams<double> &, const double *, double *, double *,
                                       const StageArgs &, cudaStream_t);
template void launch_mass<float>(const Geom &, const double *, double, double, float *, unsigned long long *,
                                 cudaStream_t);
template void launch_mass<double>(const Geom &, const double *, double, double, double *, unsigned long long *,
                                  cudaStream_t);

}  // namespace nm
