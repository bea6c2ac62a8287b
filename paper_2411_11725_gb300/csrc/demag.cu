// Demag passes (section "Demagnetization Field"): node->cell averaging fused into a pruned
// real-to-complex x transform, pruned y transforms, a z pass that fuses forward z, the pointwise
// product with the symmetric tensor spectrum and inverse z (or, for one cell layer, a y pass that
// fuses forward y, the product and inverse y), and a pruned complex-to-real x transform that writes
// Ms_c H_c per cell.
#include "demag.cuh"
#include "fft.cuh"

namespace nm {

constexpr int kFftThreads = 256;
constexpr int kMaxB = 8;                                  // radix-4 butterflies per thread per stage
constexpr int kLineBudget = 4 * kMaxB * kFftThreads;      // complex elements per block: 8192

// ---------------------------------------------------------------------------------------------
// node -> cell average times Ms: M_c = Ms_c * (1/8) sum_{i in {0,1}^3} y_{c+i}
template <typename T>
__device__ __forceinline__ T cell_M(const Geom &g, const DemagBufs<T> &b, const T *__restrict__ yc, int x, int yy,
                                    int zz)
{
    long n00 = ((long)zz * g.nn2 + yy) * g.nn1 + x;
    long n01 = n00 + g.nn1;                       // y+1
    long n10 = n00 + (long)g.nn2 * g.nn1;         // z+1
    long n11 = n10 + g.nn1;
    T s = (yc[n00] + yc[n00 + 1]) + (yc[n01] + yc[n01 + 1]) + (yc[n10] + yc[n10 + 1]) + (yc[n11] + yc[n11 + 1]);
    long c = ((long)zz * g.N2 + yy) * g.N1 + x;
    T Ms = b.Ms ? b.Ms[c] : b.Ms0;
    return Ms * T(0.125) * s;
}

// Pass 1: x transform (R2C of length P1 through a complex FFT of length Q = P1/2 on even/odd pairs).
// One block holds `rpb` cell rows (y, z) x 3 components.  CELL_IN: the input is already a cell field.
template <typename T, bool CELL_IN>
__global__ void __launch_bounds__(kFftThreads) k_x_fwd(Geom g, DemagBufs<T> b, const T *__restrict__ in, int rpb)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int nrows = g.N2 * g.N3;
    const int row0 = blockIdx.x * rpb;
    const int nr = min(rpb, nrows - row0);
    if (nr <= 0) return;
    auto M_at = [&](int c, int x, int yy, int zz) -> T {
        if (x >= g.N1) return T(0);
        if (CELL_IN) return in[c * g.cs + ((long)zz * g.N2 + yy) * g.N1 + x];
        return cell_M(g, b, in + c * g.ns, x, yy, zz);
    };
    if (g.P1 == 1) {
        for (int t = threadIdx.x; t < nr * 3; t += blockDim.x) {
            int r = t / 3, c = t - 3 * r, row = row0 + r;
            int yy = row % g.N2, zz = row / g.N2;
            b.S[c * g.s_comp + ((long)zz * g.P2 + yy) * g.Xp] = cx<T>(M_at(c, 0, yy, zz), T(0));
        }
        return;
    }
    const int Q = g.Q, ls = Q;
    const int nl = nr * 3;
    const int jmax = (g.N1 + 1) >> 1;  // pairs beyond this are zero padding
    for (int t = threadIdx.x; t < nl * Q; t += blockDim.x) {
        int j = t % Q, lc = t / Q;
        int r = lc / 3, c = lc - 3 * r, row = row0 + r;
        int yy = row % g.N2, zz = row / g.N2;
        Cx<T> v = cx<T>(T(0), T(0));
        if (j < jmax) v = cx<T>(M_at(c, 2 * j, yy, zz), M_at(c, 2 * j + 1, yy, zz));
        buf[lc * ls + j] = v;
    }
    __syncthreads();
    smem_fft<T, kMaxB>(buf, nl, ls, g.lgQ, -1, b.tw, g.twlg);
    const int wsh = g.twlg - (g.lgQ + 1);
    for (int t = threadIdx.x; t < nl * (Q + 1); t += blockDim.x) {
        int k = t % (Q + 1), lc = t / (Q + 1);
        int r = lc / 3, c = lc - 3 * r, row = row0 + r;
        int yy = row % g.N2, zz = row / g.N2;
        Cx<T> Zk = buf[lc * ls + (k == Q ? 0 : k)];
        Cx<T> Zc = conj(buf[lc * ls + (k == 0 ? 0 : Q - k)]);
        Cx<T> E = scale(Zk + Zc, T(0.5));
        Cx<T> O = scale(mul_si(Zk - Zc, -1), T(0.5));
        Cx<T> Xk = E + b.tw[k << wsh] * O;
        b.S[c * g.s_comp + ((long)zz * g.P2 + yy) * g.Xp + k] = Xk;
    }
}

// Pass 5: inverse x transform (C2R of length P1 through a complex FFT of length Q), keeping x < N1.
// Output per cell: Ms_c * H_c (or H_c when CELL_OUT, for the cell-input pipeline).
template <typename T, bool CELL_OUT>
__global__ void __launch_bounds__(kFftThreads) k_x_inv(Geom g, DemagBufs<T> b, T *__restrict__ out, int rpb)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int nrows = g.N2 * g.N3;
    const int row0 = blockIdx.x * rpb;
    const int nr = min(rpb, nrows - row0);
    if (nr <= 0) return;
    auto put = [&](int c, int x, int yy, int zz, T v) {
        long cell = ((long)zz * g.N2 + yy) * g.N1 + x;
        if (!CELL_OUT) v *= b.Ms ? b.Ms[cell] : b.Ms0;
        out[c * g.cs + cell] = v;
    };
    if (g.P1 == 1) {
        for (int t = threadIdx.x; t < nr * 3; t += blockDim.x) {
            int r = t / 3, c = t - 3 * r, row = row0 + r;
            int yy = row % g.N2, zz = row / g.N2;
            put(c, 0, yy, zz, b.S[c * g.s_comp + ((long)zz * g.P2 + yy) * g.Xp].x);
        }
        return;
    }
    const int Q = g.Q, ls = Q;
    const int nl = nr * 3;
    const int wsh = g.twlg - (g.lgQ + 1);
    for (int t = threadIdx.x; t < nl * Q; t += blockDim.x) {
        int k = t % Q, lc = t / Q;
        int r = lc / 3, c = lc - 3 * r, row = row0 + r;
        int yy = row % g.N2, zz = row / g.N2;
        const Cx<T> *src = b.S + c * g.s_comp + ((long)zz * g.P2 + yy) * g.Xp;
        Cx<T> Xk = src[k];
        Cx<T> Xc = conj(src[Q - k]);
        Cx<T> E2 = Xk + Xc;
        Cx<T> O2 = (Xk - Xc) * conj(b.tw[k << wsh]);
        buf[lc * ls + k] = E2 + mul_si(O2, 1);
    }
    __syncthreads();
    smem_fft<T, kMaxB>(buf, nl, ls, g.lgQ, +1, b.tw, g.twlg);
    const int jmax = (g.N1 + 1) >> 1;
    for (int t = threadIdx.x; t < nl * jmax; t += blockDim.x) {
        int j = t % jmax, lc = t / jmax;
        int r = lc / 3, c = lc - 3 * r, row = row0 + r;
        int yy = row % g.N2, zz = row / g.N2;
        Cx<T> v = buf[lc * ls + j];
        put(c, 2 * j, yy, zz, v.x);
        if (2 * j + 1 < g.N1) put(c, 2 * j + 1, yy, zz, v.y);
    }
}

// Passes 2 and 4: y transform of G consecutive kx columns of one (component, z) plane.
// Forward reads y < N2 (zero padding above) and writes all P2; inverse reads all P2, writes y < N2.
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_y(Geom g, DemagBufs<T> b, int G, int dir)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int P2 = g.P2, ls = P2 + 1;
    const int kx0 = blockIdx.x * G;
    Cx<T> *base = b.S + (long)blockIdx.y * P2 * g.Xp + kx0;
    const int nin = dir < 0 ? g.N2 : P2, nout = dir < 0 ? P2 : g.N2;
    for (int t = threadIdx.x; t < P2 * G; t += blockDim.x) {
        int gg = t % G, yy = t / G;
        buf[gg * ls + yy] = yy < nin ? base[(long)yy * g.Xp + gg] : cx<T>(T(0), T(0));
    }
    __syncthreads();
    smem_fft<T, kMaxB>(buf, G, ls, g.lgP2, dir, b.tw, g.twlg);
    for (int t = threadIdx.x; t < nout * G; t += blockDim.x) {
        int gg = t % G, yy = t / G;
        base[(long)yy * g.Xp + gg] = buf[gg * ls + yy];
    }
}

// H^ = N~ M^ at one frequency; N~ real symmetric, stored on the octant with the odd components'
// signs restored here (Nxy odd in ky, Nxz odd in kz, Nyz odd in both).
template <typename T>
__device__ __forceinline__ void tensor_apply(const Geom &g, const DemagBufs<T> &b, int kx, int ky, int kz, Cx<T> &mx,
                                             Cx<T> &my, Cx<T> &mz)
{
    const int h2 = g.P2 >> 1, h3 = g.P3 >> 1;
    int a2 = ky <= h2 ? ky : g.P2 - ky;
    int a3 = kz <= h3 ? kz : g.P3 - kz;
    T s2 = ky <= h2 ? T(1) : T(-1);
    T s3 = kz <= h3 ? T(1) : T(-1);
    const T *n = b.Nk + ((long)a3 * g.H2 + a2) * g.Xp + kx;
    const long tc = g.t_comp;
    T nxx = n[0], nyy = n[tc], nzz = n[2 * tc];
    T nxy = n[3 * tc] * s2, nxz = n[4 * tc] * s3, nyz = n[5 * tc] * (s2 * s3);
    Cx<T> hx = cx<T>(nxx * mx.x + nxy * my.x + nxz * mz.x, nxx * mx.y + nxy * my.y + nxz * mz.y);
    Cx<T> hy = cx<T>(nxy * mx.x + nyy * my.x + nyz * mz.x, nxy * mx.y + nyy * my.y + nyz * mz.y);
    Cx<T> hz = cx<T>(nxz * mx.x + nyz * my.x + nzz * mz.x, nxz * mx.y + nyz * my.y + nzz * mz.y);
    mx = hx; my = hy; mz = hz;
}

// Pass 3 (N3 > 1): for G kx columns and KY ky rows: forward z (N3 non-zero inputs), tensor product,
// inverse z keeping z < N3.
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_z_conv(Geom g, DemagBufs<T> b, int G, int KY)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int P3 = g.P3, ls = P3 + 1;
    const int kx0 = blockIdx.x * G, ky0 = blockIdx.y * KY;
    const int nky = min(KY, g.P2 - ky0);
    const int nl = nky * 3 * G;
    // line lc = (kyl * 3 + c) * G + gg
    for (int t = threadIdx.x; t < nl * P3; t += blockDim.x) {
        int gg = t % G, r = t / G;
        int c = r % 3; r /= 3;
        int kyl = r % nky, zz = r / nky;
        int lc = (kyl * 3 + c) * G + gg;
        buf[lc * ls + zz] = zz < g.N3 ? b.S[c * g.s_comp + ((long)zz * g.P2 + ky0 + kyl) * g.Xp + kx0 + gg]
                                      : cx<T>(T(0), T(0));
    }
    __syncthreads();
    smem_fft<T, kMaxB>(buf, nl, ls, g.lgP3, -1, b.tw, g.twlg);
    for (int t = threadIdx.x; t < nky * G * P3; t += blockDim.x) {
        int gg = t % G, r = t / G;
        int kyl = r % nky, kz = r / nky;
        Cx<T> *px = buf + ((kyl * 3 + 0) * G + gg) * ls + kz;
        Cx<T> *py = buf + ((kyl * 3 + 1) * G + gg) * ls + kz;
        Cx<T> *pz = buf + ((kyl * 3 + 2) * G + gg) * ls + kz;
        Cx<T> mx = *px, my = *py, mz = *pz;
        tensor_apply(g, b, kx0 + gg, ky0 + kyl, kz, mx, my, mz);
        *px = mx; *py = my; *pz = mz;
    }
    __syncthreads();
    smem_fft<T, kMaxB>(buf, nl, ls, g.lgP3, +1, b.tw, g.twlg);
    for (int t = threadIdx.x; t < nl * g.N3; t += blockDim.x) {
        int gg = t % G, r = t / G;
        int c = r % 3; r /= 3;
        int kyl = r % nky, zz = r / nky;
        int lc = (kyl * 3 + c) * G + gg;
        b.S[c * g.s_comp + ((long)zz * g.P2 + ky0 + kyl) * g.Xp + kx0 + gg] = buf[lc * ls + zz];
    }
}

// Single-layer variant (N3 == 1, P3 == 1): forward y, tensor product at kz = 0, inverse y.
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_y_conv(Geom g, DemagBufs<T> b, int G)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int P2 = g.P2, ls = P2 + 1;
    const int kx0 = blockIdx.x * G;
    const int nl = 3 * G;  // lc = c * G + gg
    for (int t = threadIdx.x; t < nl * P2; t += blockDim.x) {
        int gg = t % G, r = t / G;
        int c = r % 3, yy = r / 3;
        buf[(c * G + gg) * ls + yy] = yy < g.N2 ? b.S[c * g.s_comp + (long)yy * g.Xp + kx0 + gg] : cx<T>(T(0), T(0));
    }
    __syncthreads();
    smem_fft<T, kMaxB>(buf, nl, ls, g.lgP2, -1, b.tw, g.twlg);
    for (int t = threadIdx.x; t < G * P2; t += blockDim.x) {
        int gg = t % G, ky = t / G;
        Cx<T> *px = buf + (0 * G + gg) * ls + ky;
        Cx<T> *py = buf + (1 * G + gg) * ls + ky;
        Cx<T> *pz = buf + (2 * G + gg) * ls + ky;
        Cx<T> mx = *px, my = *py, mz = *pz;
        tensor_apply(g, b, kx0 + gg, ky, 0, mx, my, mz);
        *px = mx; *py = my; *pz = mz;
    }
    __syncthreads();
    smem_fft<T, kMaxB>(buf, nl, ls, g.lgP2, +1, b.tw, g.twlg);
    for (int t = threadIdx.x; t < nl * g.N2; t += blockDim.x) {
        int gg = t % G, r = t / G;
        int c = r % 3, yy = r / 3;
        b.S[c * g.s_comp + (long)yy * g.Xp + kx0 + gg] = buf[(c * G + gg) * ls + yy];
    }
}

// ---------------------------------------------------------------------------------------------
// host side: launch shapes (lines per block bounded by the FFT engine's per-thread budget)
void demag_init_attributes()
{
    static bool done = false;
    if (done) return;
    const int lim = 200 * 1024;
    const void *fns[] = {(const void *)k_x_fwd<float, false>, (const void *)k_x_fwd<float, true>,
                         (const void *)k_x_fwd<double, false>, (const void *)k_x_fwd<double, true>,
                         (const void *)k_x_inv<float, false>, (const void *)k_x_inv<float, true>,
                         (const void *)k_x_inv<double, false>, (const void *)k_x_inv<double, true>,
                         (const void *)k_y<float>, (const void *)k_y<double>,
                         (const void *)k_z_conv<float>, (const void *)k_z_conv<double>,
                         (const void *)k_y_conv<float>, (const void *)k_y_conv<double>};
    for (const void *f : fns) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    done = true;
}

static int pow2_floor(int v)
{
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

template <typename T, bool CELL>
static void run_pipeline(const Geom &g, const DemagBufs<T> &b, const T *in, T *out, cudaStream_t st)
{
    const int nrows = g.N2 * g.N3;
    const size_t cs = sizeof(Cx<T>);
    // pass 1
    {
        int Q = g.P1 == 1 ? 1 : g.Q;
        int rpb = kLineBudget / (3 * Q);
        rpb = rpb < 1 ? 1 : rpb;
        int cap = (int)((96 * 1024) / (3 * Q * cs));
        rpb = rpb > cap ? cap : rpb;
        if (rpb < 1) rpb = 1;
        rpb = rpb > nrows ? nrows : rpb;
        size_t sm = g.P1 == 1 ? 0 : (size_t)rpb * 3 * Q * cs;
        auto fn = k_x_fwd<T, CELL>;
        fn<<<div_up(nrows, rpb), kFftThreads, sm, st>>>(g, b, in, rpb);
    }
    // passes 2-4
    if (g.N3 > 1) {
        if (g.P2 > 1) {
            int G = pow2_floor(kLineBudget / g.P2);
            G = G > 16 ? 16 : G;
            size_t sm = (size_t)G * (g.P2 + 1) * cs;
            k_y<T><<<dim3(g.Xp / G, 3 * g.N3), kFftThreads, sm, st>>>(g, b, G, -1);
        }
        {
            int G = 16;
            int KY = pow2_floor(kLineBudget / (3 * G * g.P3));
            KY = KY < 1 ? 1 : KY;
            KY = KY > g.P2 ? pow2_floor(g.P2) : KY;
            size_t sm = (size_t)3 * G * KY * (g.P3 + 1) * cs;
            k_z_conv<T><<<dim3(g.Xp / G, div_up(g.P2, KY)), kFftThreads, sm, st>>>(g, b, G, KY);
        }
        if (g.P2 > 1) {
            int G = pow2_floor(kLineBudget / g.P2);
            G = G > 16 ? 16 : G;
            size_t sm = (size_t)G * (g.P2 + 1) * cs;
            k_y<T><<<dim3(g.Xp / G, 3 * g.N3), kFftThreads, sm, st>>>(g, b, G, +1);
        }
    } else {
        int G = pow2_floor(kLineBudget / (3 * g.P2));
        G = G > 16 ? 16 : G;
        G = G < 1 ? 1 : G;
        size_t sm = (size_t)3 * G * (g.P2 + 1) * cs;
        k_y_conv<T><<<g.Xp / G, kFftThreads, sm, st>>>(g, b, G);
    }
    // pass 5
    {
        int Q = g.P1 == 1 ? 1 : g.Q;
        int rpb = kLineBudget / (3 * Q);
        int cap = (int)((96 * 1024) / (3 * Q * cs));
        rpb = rpb > cap ? cap : rpb;
        if (rpb < 1) rpb = 1;
        rpb = rpb > nrows ? nrows : rpb;
        size_t sm = g.P1 == 1 ? 0 : (size_t)rpb * 3 * Q * cs;
        auto fn = k_x_inv<T, CELL>;
        fn<<<div_up(nrows, rpb), kFftThreads, sm, st>>>(g, b, out, rpb);
    }
}

template <typename T>
void demag_forward(const Geom &g, const DemagBufs<T> &b, const T *y, T *MsH, cudaStream_t st)
{
    run_pipeline<T, false>(g, b, y, MsH, st);
}

template <typename T>
void demag_cells(const Geom &g, const DemagBufs<T> &b, const T *M, T *H, cudaStream_t st)
{
    run_pipeline<T, true>(g, b, M, H, st);
}

template void demag_forward<float>(const Geom &, const DemagBufs<float> &, const float *, float *, cudaStream_t);
template void demag_forward<double>(const Geom &, const DemagBufs<double> &, const double *, double *, cudaStream_t);
template void demag_cells<float>(const Geom &, const DemagBufs<float> &, const float *, float *, cudaStream_t);
template void demag_cells<double>(const Geom &, const DemagBufs<double> &, const double *, double *, cudaStream_t);

}  // namespace nm
