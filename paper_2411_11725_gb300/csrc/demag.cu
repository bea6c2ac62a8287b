// Demag passes (section "Demagnetization Field"): node->cell averaging fused into a pruned
// real-to-complex x transform, pruned y transforms, a z pass that fuses forward z, the pointwise
// product with the symmetric tensor spectrum and inverse z (or, for one cell layer, a y pass that
// fuses forward y, the product and inverse y), and a pruned complex-to-real x transform that writes
// Ms_c H_c per cell.
//
// The x passes read their input in the first FFT stage straight from global memory (the zero padding
// is never read); the y and z passes stage their strided tiles in shared memory with cp.async (all
// copies of a tile in flight at once).  Every pass writes its output from the last FFT stage straight
// to global memory, and only the part that later passes read.
#include "demag.cuh"
#include "fft.cuh"

namespace nm {

constexpr int kFftThreads = 256;

// ---------------------------------------------------------------------------------------------
// node -> cell average times Ms for the cell pair (x, x+1) of one cell row:
// M_c = Ms_c * (1/8) sum_{i in {0,1}^3} y_{c+i}
template <typename T>
__device__ __forceinline__ Cx<T> cell_M_pair(const Geom &g, const DemagBufs<T> &b, const T *__restrict__ yc,
                                             long r00, long c0, int x)
{
    const long r01 = r00 + g.nn1;
    const long r10 = r00 + (long)g.nn2 * g.nn1;
    const long r11 = r10 + g.nn1;
    const T a0 = (yc[r00] + yc[r01]) + (yc[r10] + yc[r11]);
    const T a1 = (yc[r00 + 1] + yc[r01 + 1]) + (yc[r10 + 1] + yc[r11 + 1]);
    const T Ms0 = b.Ms ? b.Ms[c0] : b.Ms0;
    T m0 = Ms0 * T(0.125) * (a0 + a1), m1 = T(0);
    if (x + 1 < g.N1) {
        const T a2 = (yc[r00 + 2] + yc[r01 + 2]) + (yc[r10 + 2] + yc[r11 + 2]);
        const T Ms1 = b.Ms ? b.Ms[c0 + 1] : b.Ms0;
        m1 = Ms1 * T(0.125) * (a1 + a2);
    }
    return cx<T>(m0, m1);
}

// Line L of the x passes is (cell row, component) = (L / 3, L % 3); cell row = zz * N2 + yy.
struct XLine {
    int c, yy, zz, row;
};
__device__ __forceinline__ XLine x_line(const Geom &g, int L)
{
    XLine x;
    x.row = L / 3;
    x.c = L - 3 * x.row;
    x.zz = (int)g.n2f.div((unsigned)x.row);
    x.yy = x.row - x.zz * g.N2;
    return x;
}

// Pass 1: x transform (R2C of length P1 via a complex FFT of length Q = P1/2 on even/odd pairs).
// One block holds `lpb` consecutive lines.  CELL_IN: the input is already a cell field.
template <typename T, bool CELL_IN>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 2 : 1) k_x_fwd(Geom g, DemagBufs<T> b, const T *__restrict__ in, int lpb)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int nlines = 3 * g.N2 * g.N3;
    const int l0 = blockIdx.x * lpb;
    const int nl = min(lpb, nlines - l0);
    if (nl <= 0) return;
    auto pair = [&](const XLine &xl, int x) -> Cx<T> {
        const long c0 = (long)xl.row * g.N1 + x;
        if (CELL_IN) {
            const T *p = in + xl.c * g.cs + c0;
            return cx<T>(p[0], x + 1 < g.N1 ? p[1] : T(0));
        }
        const long r00 = ((long)xl.zz * g.nn2 + xl.yy) * g.nn1 + x;
        return cell_M_pair(g, b, in + xl.c * g.ns, r00, c0, x);
    };
    if (g.P1 == 1) {
        for (int t = threadIdx.x; t < nl; t += blockDim.x) {
            const XLine xl = x_line(g, l0 + t);
            b.S[xl.c * g.s_comp + ((long)xl.zz * g.P2 + xl.yy) * g.Xp] = cx<T>(pair(xl, 0).x, T(0));
        }
        return;
    }
    const int Q = g.Q, lsz = padded_len(Q);
    auto src = [&](int l, int i) -> Cx<T> { return pair(x_line(g, l0 + l), 2 * i); };
    auto sm = [&](int l, int i) { return l * lsz + pad16(i); };
    auto dst = [&](int l, int i, Cx<T> v) { buf[l * lsz + pad16(i)] = v; };
    fft_lines<T, false, false, true>(buf, FastDiv((unsigned)nl), g.lgQ, -1, b.tw, g.twlg, (g.N1 + 1) >> 1, Q, src,
                                     sm, dst);
    // X_k = (Z_k + conj Z_{Q-k})/2 - (i/2) W^k (Z_k - conj Z_{Q-k}),  W = e^{-2 pi i / P1},  k = 0..Q
    const int wsh = g.twlg - (g.lgQ + 1);
    const FastDiv qf((unsigned)(Q + 1));
    for (int t = threadIdx.x; t < nl * (Q + 1); t += blockDim.x) {
        const int l = (int)qf.div((unsigned)t), k = t - l * (Q + 1);
        const XLine xl = x_line(g, l0 + l);
        const Cx<T> Zk = buf[l * lsz + pad16(k == Q ? 0 : k)];
        const Cx<T> Zc = conj(buf[l * lsz + pad16(k == 0 ? 0 : Q - k)]);
        const Cx<T> E = scale(Zk + Zc, T(0.5));
        const Cx<T> O = scale(mul_si(Zk - Zc, -1), T(0.5));
        b.S[xl.c * g.s_comp + ((long)xl.zz * g.P2 + xl.yy) * g.Xp + k] = E + b.tw[k << wsh] * O;
    }
}

// Pass 5: inverse x transform (C2R of length P1 via a complex FFT of length Q), keeping x < N1.
// Lines as in pass 1.  Output per cell: Ms_c H_c (or H_c when CELL_OUT).
template <typename T, bool CELL_OUT>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 2 : 1) k_x_inv(Geom g, DemagBufs<T> b, T *__restrict__ out, int lpb)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int nlines = 3 * g.N2 * g.N3;
    const int l0 = blockIdx.x * lpb;
    const int nl = min(lpb, nlines - l0);
    if (nl <= 0) return;
    auto put = [&](int c, long cell, T v) {
        if (!CELL_OUT) v *= b.Ms ? b.Ms[cell] : b.Ms0;
        out[c * g.cs + cell] = v;
    };
    if (g.P1 == 1) {
        for (int t = threadIdx.x; t < nl; t += blockDim.x) {
            const XLine xl = x_line(g, l0 + t);
            put(xl.c, (long)xl.row * g.N1, b.S[xl.c * g.s_comp + ((long)xl.zz * g.P2 + xl.yy) * g.Xp].x);
        }
        return;
    }
    const int Q = g.Q, lsz = padded_len(Q);
    const int wsh = g.twlg - (g.lgQ + 1);
    // Z_k = (X_k + conj X_{Q-k}) + i e^{2 pi i k / P1} (X_k - conj X_{Q-k}), k < Q
    auto src = [&](int l, int k) -> Cx<T> {
        const XLine xl = x_line(g, l0 + l);
        const Cx<T> *s = b.S + xl.c * g.s_comp + ((long)xl.zz * g.P2 + xl.yy) * g.Xp;
        const Cx<T> Xk = s[k], Xc = conj(s[Q - k]);
        return (Xk + Xc) + mul_si((Xk - Xc) * conj(b.tw[k << wsh]), 1);
    };
    auto sm = [&](int l, int i) { return l * lsz + pad16(i); };
    auto dst = [&](int l, int j, Cx<T> v) {
        const XLine xl = x_line(g, l0 + l);
        const long cell = (long)xl.row * g.N1 + 2 * j;
        put(xl.c, cell, v.x);
        if (2 * j + 1 < g.N1) put(xl.c, cell + 1, v.y);
    };
    fft_lines<T, false, false, false>(buf, FastDiv((unsigned)nl), g.lgQ, +1, b.tw, g.twlg, Q, (g.N1 + 1) >> 1, src,
                                      sm, dst);
}

// Passes 2 and 4: y transform of G consecutive kx columns of one (component, z) plane, in place.
// Forward reads y < N2 (zero padding above) and writes all P2; inverse reads all P2, writes y < N2.
// The rows are staged with cp.async (all in flight at once), the last stage writes global memory.
template <typename T>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 2 : 1) k_y(Geom g, DemagBufs<T> b, int G, int dir)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *base = b.S + (long)blockIdx.y * g.P2 * g.Xp + blockIdx.x * G;
    const int nin = dir < 0 ? g.N2 : g.P2, nout = dir < 0 ? g.P2 : g.N2;
    const int Xp = g.Xp;
    const int rowb = G * (int)sizeof(Cx<T>);
    const int cb = rowb >= 16 ? 16 : rowb;  // bytes per async copy
    const int lcpr = __ffs(rowb / cb) - 1;  // copies per row is a power of two
    for (int t = threadIdx.x; t < (nin << lcpr); t += blockDim.x) {
        const int y = t >> lcpr, ch = t - (y << lcpr);
        char *d = (char *)(buf + pad16(y) * G) + ch * cb;
        const char *s = (const char *)(base + y * Xp) + ch * cb;
        if (cb == 16) cp_async16(d, s);
        else cp_async8(d, s);
    }
    cp_async_wait_all();
    __syncthreads();
    auto sm = [&](int l, int i) { return pad16(i) * G + l; };
    auto sm_src = [&](int l, int i) { return buf[pad16(i) * G + l]; };
    auto dst = [&](int l, int i, Cx<T> v) { base[i * Xp + l] = v; };
    fft_lines<T, true, true, false>(buf, FastDiv((unsigned)G), g.lgP2, dir, b.tw, g.twlg, nin, nout, sm_src, sm, dst);
}

// The six real tensor components at octant frequency (kx, a2, kz), with the sign of the odd ones in
// kz restored (Nxz odd in kz, Nyz odd in kz); the y parity is applied by the caller (s2).
template <typename T>
struct Ten6 {
    T xx, yy, zz, xy, xz, yz;
};
template <typename T>
__device__ __forceinline__ Ten6<T> tensor_at(const Geom &g, const DemagBufs<T> &b, int kx, int a2, int kz)
{
    const int h3 = g.P3 >> 1;
    const int a3 = kz <= h3 ? kz : g.P3 - kz;
    const T s3 = kz <= h3 ? T(1) : T(-1);
    const T *n = b.Nk + ((long)a3 * g.H2 + a2) * g.Xp + kx;
    const long tc = g.t_comp;
    Ten6<T> t;
    t.xx = n[0]; t.yy = n[tc]; t.zz = n[2 * tc];
    t.xy = n[3 * tc]; t.xz = n[4 * tc] * s3; t.yz = n[5 * tc] * s3;
    return t;
}
// H^ = N~ M^ with N~ real symmetric; s2 = -1 on the mirrored frequency P2 - a2 (Nxy and Nyz odd in ky)
template <typename T>
__device__ __forceinline__ void tensor_mul(const Ten6<T> &t, T s2, Cx<T> *px, Cx<T> *py, Cx<T> *pz)
{
    const Cx<T> mx = *px, my = *py, mz = *pz;
    const T nxy = t.xy * s2, nyz = t.yz * s2;
    *px = cx<T>(t.xx * mx.x + nxy * my.x + t.xz * mz.x, t.xx * mx.y + nxy * my.y + t.xz * mz.y);
    *py = cx<T>(nxy * mx.x + t.yy * my.x + nyz * mz.x, nxy * mx.y + t.yy * my.y + nyz * mz.y);
    *pz = cx<T>(t.xz * mx.x + nyz * my.x + t.zz * mz.x, t.xz * mx.y + nyz * my.y + t.zz * mz.y);
}

// Pass 3 (N3 > 1): G kx columns x KY octant rows a2 (each with its mirror P2 - a2, so the tensor is
// read once): forward z (N3 non-zero inputs), tensor product, inverse z keeping z < N3.
// Rows r < KY are ky = a2_0 + r, rows KY + r are ky = P2 - (a2_0 + r) (present when 0 < a2 < P2/2).
// Lines l = (c * 2KY + r) * G + g, innermost in shared memory.
template <typename T>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 2 : 1) k_z_conv(Geom g, DemagBufs<T> b, int G, int KY)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int kx0 = blockIdx.x * G, a20 = blockIdx.y * KY;
    const int R2 = 2 * KY, nl = 3 * R2 * G;
    const int h2 = g.P2 >> 1;
    auto row_ky = [&](int r) -> int {  // -1: row absent
        const int a2 = a20 + (r < KY ? r : r - KY);
        if (a2 >= g.H2) return -1;
        if (r < KY) return a2;
        return (a2 > 0 && a2 < h2) ? g.P2 - a2 : -1;
    };
    auto gaddr = [&](int c, int ky, int z) -> long {
        return c * g.s_comp + ((long)z * g.P2 + ky) * g.Xp + kx0;
    };
    {
        const int rowb = G * (int)sizeof(Cx<T>);
        const int cb = rowb >= 16 ? 16 : rowb, lcpr = __ffs(rowb / cb) - 1, lR2 = __ffs(R2) - 1;
        const int nrow = g.N3 * 3 * R2;
        for (int t = threadIdx.x; t < (nrow << lcpr); t += blockDim.x) {
            const int rr = t >> lcpr, ch = t - (rr << lcpr);
            const int r = rr & (R2 - 1), cz = rr >> lR2, z = cz / 3, c = cz - 3 * z;
            const int ky = row_ky(r);
            if (ky < 0) continue;
            char *d = (char *)(buf + pad16(z) * nl + (c * R2 + r) * G) + ch * cb;
            const char *s = (const char *)(b.S + gaddr(c, ky, z)) + ch * cb;
            if (cb == 16) cp_async16(d, s);
            else cp_async8(d, s);
        }
        cp_async_wait_all();
        __syncthreads();
    }
    const FastDiv nlf((unsigned)nl);
    auto sm = [&](int l, int i) { return pad16(i) * nl + l; };
    auto sm_src = [&](int l, int i) { return buf[pad16(i) * nl + l]; };
    auto sm_dst = [&](int l, int i, Cx<T> v) { buf[pad16(i) * nl + l] = v; };
    fft_lines<T, true, true, true>(buf, nlf, g.lgP3, -1, b.tw, g.twlg, g.N3, g.P3, sm_src, sm, sm_dst);
    const int npts = KY * G * g.P3;
    const int lG = __ffs(G) - 1, lKY = __ffs(KY) - 1;
    for (int t = threadIdx.x; t < npts; t += blockDim.x) {
        const int gg = t & (G - 1), q = t >> lG, rr = q & (KY - 1), kz = q >> lKY;
        const int a2 = a20 + rr;
        if (a2 >= g.H2) continue;
        const Ten6<T> ten = tensor_at(g, b, kx0 + gg, a2, kz);
        Cx<T> *p = buf + pad16(kz) * nl + rr * G + gg;
        tensor_mul(ten, T(1), p, p + R2 * G, p + 2 * R2 * G);
        if (a2 > 0 && a2 < h2) {
            Cx<T> *pm = p + KY * G;
            tensor_mul(ten, T(-1), pm, pm + R2 * G, pm + 2 * R2 * G);
        }
    }
    __syncthreads();
    auto dst = [&](int l, int z, Cx<T> v) {
        const int gg = l & (G - 1), q = l >> lG, r = q & (R2 - 1), c = q >> (lKY + 1);
        const int ky = row_ky(r);
        if (ky >= 0) b.S[gaddr(c, ky, z) + gg] = v;
    };
    fft_lines<T, true, true, false>(buf, nlf, g.lgP3, +1, b.tw, g.twlg, g.P3, g.N3, sm_src, sm, dst);
}

// Single-layer variant (N3 == 1, P3 == 1): forward y, tensor product at kz = 0 (each octant row a2
// read once and applied to ky = a2 and P2 - a2), inverse y.  Lines l = c * G + g.
template <typename T>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 2 : 1) k_y_conv(Geom g, DemagBufs<T> b, int G)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int kx0 = blockIdx.x * G;
    const int nl = 3 * G;
    const int h2 = g.P2 >> 1;
    auto gaddr = [&](int c, int y) -> long { return c * g.s_comp + (long)y * g.Xp + kx0; };
    {
        const int rowb = G * (int)sizeof(Cx<T>);
        const int cb = rowb >= 16 ? 16 : rowb, lcpr = __ffs(rowb / cb) - 1;
        const int nrow = g.N2 * 3;
        for (int t = threadIdx.x; t < (nrow << lcpr); t += blockDim.x) {
            const int rr = t >> lcpr, ch = t - (rr << lcpr);
            const int y = rr / 3, c = rr - 3 * y;
            char *d = (char *)(buf + pad16(y) * nl + c * G) + ch * cb;
            const char *s = (const char *)(b.S + gaddr(c, y)) + ch * cb;
            if (cb == 16) cp_async16(d, s);
            else cp_async8(d, s);
        }
        cp_async_wait_all();
        __syncthreads();
    }
    const FastDiv nlf((unsigned)nl);
    auto sm = [&](int l, int i) { return pad16(i) * nl + l; };
    auto sm_src = [&](int l, int i) { return buf[pad16(i) * nl + l]; };
    auto sm_dst = [&](int l, int i, Cx<T> v) { buf[pad16(i) * nl + l] = v; };
    fft_lines<T, true, true, true>(buf, nlf, g.lgP2, -1, b.tw, g.twlg, g.N2, g.P2, sm_src, sm, sm_dst);
    const int lG = __ffs(G) - 1;
    for (int t = threadIdx.x; t < G * g.H2; t += blockDim.x) {
        const int gg = t & (G - 1), a2 = t >> lG;
        const Ten6<T> ten = tensor_at(g, b, kx0 + gg, a2, 0);
        Cx<T> *p = buf + pad16(a2) * nl + gg;
        tensor_mul(ten, T(1), p, p + G, p + 2 * G);
        if (a2 > 0 && a2 < h2) {
            Cx<T> *pm = buf + pad16(g.P2 - a2) * nl + gg;
            tensor_mul(ten, T(-1), pm, pm + G, pm + 2 * G);
        }
    }
    __syncthreads();
    auto dst = [&](int l, int y, Cx<T> v) {
        const int gg = l & (G - 1), c = l >> lG;
        b.S[gaddr(c, y) + gg] = v;
    };
    fft_lines<T, true, true, false>(buf, nlf, g.lgP2, +1, b.tw, g.twlg, g.P2, g.N2, sm_src, sm, dst);
}

// ---------------------------------------------------------------------------------------------
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

static int pow2_floor(long v)
{
    int p = 1;
    while (2L * p <= v) p *= 2;
    return p;
}

// Launch shapes: every block transforms at most fft_regs<T>() * kFftThreads complex values.
template <typename T>
DemagPlan demag_plan(const Geom &g)
{
    DemagPlan p{};
    p.ok = true;
    const size_t cs = sizeof(Cx<T>);
    const long budget = (long)fft_regs<T>() * kFftThreads;
    const int nlines = 3 * g.N2 * g.N3;
    {
        const int Q = g.P1 == 1 ? 1 : g.Q;
        int lpb = (int)(budget / Q);
        if (lpb < 1) p.ok = false;
        lpb = lpb < 1 ? 1 : lpb;
        lpb = lpb > 48 ? 48 : lpb;
        lpb = lpb > nlines ? nlines : lpb;
        p.x_lpb = lpb;
        p.x_threads = kFftThreads;
        p.x_smem = g.P1 == 1 ? 0 : (size_t)lpb * padded_len(Q) * cs;
    }
    if (g.N3 > 1) {
        int G = pow2_floor(budget / g.P2);
        if ((long)G * g.P2 > budget) p.ok = false;
        G = G > 16 ? 16 : G;
        p.y_G = G;
        p.y_threads = kFftThreads;
        p.y_smem = (size_t)padded_len(g.P2) * G * cs;
        int Gz = pow2_floor(budget / (6L * g.P3));
        if (6L * Gz * g.P3 > budget) p.ok = false;
        Gz = Gz > 16 ? 16 : Gz;
        int KY = pow2_floor(budget / (6L * Gz * g.P3));
        KY = KY > g.H2 ? pow2_floor(g.H2) : KY;
        p.z_G = Gz;
        p.z_KY = KY;
        p.z_threads = kFftThreads;
        p.z_smem = (size_t)padded_len(g.P3) * 6 * KY * Gz * cs;
    } else {
        int G = pow2_floor(budget / (3L * g.P2));
        if (3L * G * g.P2 > budget) p.ok = false;
        G = G > 16 ? 16 : G;
        p.yc_G = G;
        p.yc_threads = kFftThreads;
        p.yc_smem = (size_t)padded_len(g.P2) * 3 * G * cs;
    }
    // the kx grouping divides Xp (a multiple of 16)
    const int Gmax = g.N3 > 1 ? (p.y_G > p.z_G ? p.y_G : p.z_G) : p.yc_G;
    if (g.Xp % Gmax != 0) p.ok = false;
    if (p.x_smem > 200 * 1024 || p.y_smem > 200 * 1024 || p.z_smem > 200 * 1024 || p.yc_smem > 200 * 1024)
        p.ok = false;
    return p;
}

template <typename T, bool CELL>
static void run_pipeline(const Geom &g, const DemagBufs<T> &b, const T *in, T *out, cudaStream_t st)
{
    const DemagPlan p = demag_plan<T>(g);
    if (!p.ok) return;
    const int nlines = 3 * g.N2 * g.N3;
    k_x_fwd<T, CELL><<<div_up(nlines, p.x_lpb), p.x_threads, p.x_smem, st>>>(g, b, in, p.x_lpb);
    b.mark("demag_x_fwd");
    if (g.N3 > 1) {
        if (g.P2 > 1) {
            k_y<T><<<dim3(g.Xp / p.y_G, 3 * g.N3), p.y_threads, p.y_smem, st>>>(g, b, p.y_G, -1);
            b.mark("demag_y_fwd");
        }
        k_z_conv<T><<<dim3(g.Xp / p.z_G, div_up(g.H2, p.z_KY)), p.z_threads, p.z_smem, st>>>(g, b, p.z_G, p.z_KY);
        b.mark("demag_z_conv");
        if (g.P2 > 1) {
            k_y<T><<<dim3(g.Xp / p.y_G, 3 * g.N3), p.y_threads, p.y_smem, st>>>(g, b, p.y_G, +1);
            b.mark("demag_y_inv");
        }
    } else {
        k_y_conv<T><<<g.Xp / p.yc_G, p.yc_threads, p.yc_smem, st>>>(g, b, p.yc_G);
        b.mark("demag_y_conv");
    }
    k_x_inv<T, CELL><<<div_up(nlines, p.x_lpb), p.x_threads, p.x_smem, st>>>(g, b, out, p.x_lpb);
    b.mark("demag_x_inv");
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

template DemagPlan demag_plan<float>(const Geom &);
template DemagPlan demag_plan<double>(const Geom &);
template void demag_forward<float>(const Geom &, const DemagBufs<float> &, const float *, float *, cudaStream_t);
template void demag_forward<double>(const Geom &, const DemagBufs<double> &, const double *, double *, cudaStream_t);
template void demag_cells<float>(const Geom &, const DemagBufs<float> &, const float *, float *, cudaStream_t);
template void demag_cells<double>(const Geom &, const DemagBufs<double> &, const double *, double *, cudaStream_t);

}  // namespace nm
