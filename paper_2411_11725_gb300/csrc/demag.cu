// Demag passes (section "Demagnetization Field"): node->cell averaging fused into a pruned
// real-to-complex x transform, pruned y transforms, a z pass that fuses forward z, the pointwise
// product with the symmetric tensor spectrum and inverse z (or, for one cell layer, a y pass that
// fuses forward y, the product and inverse y), and a pruned complex-to-real x transform that writes
// Ms_c H_c per cell.
//
// Every pass reads its input in the first FFT stage straight from global memory (the zero padding is
// never read) and writes its output from the last stage straight to global memory (outputs that no
// later pass needs are never written); shared memory only carries the exchanges between stages.
#include "demag.cuh"
#include "fft.cuh"

namespace nm {

// ---------------------------------------------------------------------------------------------
// node -> cell average times Ms for the cell pair (x, x+1) of one cell row:
// M_c = Ms_c * (1/8) sum_{i in {0,1}^3} y_{c+i}
template <typename T>
__device__ __forceinline__ Cx<T> cell_M_pair(const Geom &g, const DemagBufs<T> &b, const T *__restrict__ yc, int x,
                                             int yy, int zz)
{
    const long r00 = ((long)zz * g.nn2 + yy) * g.nn1 + x;
    const long r01 = r00 + g.nn1;
    const long r10 = r00 + (long)g.nn2 * g.nn1;
    const long r11 = r10 + g.nn1;
    const long c0 = ((long)zz * g.N2 + yy) * g.N1 + x;
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

// Pass 1: x transform (R2C of length P1 via a complex FFT of length Q = P1/2 on even/odd pairs).
// Lines are (cell row (y, z), component) pairs, line index = 3 * row + component; one block holds
// `lpb` consecutive lines.  CELL_IN: the input is already a cell field.
template <typename T, bool CELL_IN>
__global__ void __launch_bounds__(512) k_x_fwd(Geom g, DemagBufs<T> b, const T *__restrict__ in, int lpb)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int nlines = 3 * g.N2 * g.N3;
    const int l0 = blockIdx.x * lpb;
    const int nl = min(lpb, nlines - l0);
    if (nl <= 0) return;
    auto pair = [&](int c, int x, int yy, int zz) -> Cx<T> {
        if (CELL_IN) {
            const T *p = in + c * g.cs + ((long)zz * g.N2 + yy) * g.N1 + x;
            return cx<T>(p[0], x + 1 < g.N1 ? p[1] : T(0));
        }
        return cell_M_pair(g, b, in + c * g.ns, x, yy, zz);
    };
    if (g.P1 == 1) {
        for (int t = threadIdx.x; t < nl; t += blockDim.x) {
            const int L = l0 + t, row = L / 3, c = L - 3 * row;
            const int yy = row % g.N2, zz = row / g.N2;
            b.S[c * g.s_comp + ((long)zz * g.P2 + yy) * g.Xp] = cx<T>(pair(c, 0, yy, zz).x, T(0));
        }
        return;
    }
    const int Q = g.Q, lsz = padded_len(Q);
    auto src = [&](int l, int i) -> Cx<T> {
        const int L = l0 + l, row = L / 3, c = L - 3 * row;
        return pair(c, 2 * i, row % g.N2, row / g.N2);
    };
    auto sm = [&](int l, int i) { return l * lsz + pad16(i); };
    auto dst = [&](int l, int i, Cx<T> v) { buf[l * lsz + pad16(i)] = v; };
    fft_lines<T, false, false, true>(buf, nl, g.lgQ, -1, b.tw, g.twlg, (g.N1 + 1) >> 1, Q, src, sm, dst);
    // X_k = (Z_k + conj Z_{Q-k})/2 - (i/2) W^k (Z_k - conj Z_{Q-k}),  W = e^{-2 pi i / P1},  k = 0..Q
    const int wsh = g.twlg - (g.lgQ + 1);
    for (int t = threadIdx.x; t < nl * (Q + 1); t += blockDim.x) {
        const int k = t % (Q + 1), l = t / (Q + 1);
        const int L = l0 + l, row = L / 3, c = L - 3 * row;
        const int yy = row % g.N2, zz = row / g.N2;
        const Cx<T> Zk = buf[l * lsz + pad16(k == Q ? 0 : k)];
        const Cx<T> Zc = conj(buf[l * lsz + pad16(k == 0 ? 0 : Q - k)]);
        const Cx<T> E = scale(Zk + Zc, T(0.5));
        const Cx<T> O = scale(mul_si(Zk - Zc, -1), T(0.5));
        b.S[c * g.s_comp + ((long)zz * g.P2 + yy) * g.Xp + k] = E + b.tw[k << wsh] * O;
    }
}

// Pass 5: inverse x transform (C2R of length P1 via a complex FFT of length Q), keeping x < N1.
// Lines as in pass 1.  Output per cell: Ms_c H_c (or H_c when CELL_OUT).
template <typename T, bool CELL_OUT>
__global__ void __launch_bounds__(512) k_x_inv(Geom g, DemagBufs<T> b, T *__restrict__ out, int lpb)
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
            const int L = l0 + t, row = L / 3, c = L - 3 * row;
            const int yy = row % g.N2, zz = row / g.N2;
            put(c, ((long)zz * g.N2 + yy) * g.N1, b.S[c * g.s_comp + ((long)zz * g.P2 + yy) * g.Xp].x);
        }
        return;
    }
    const int Q = g.Q, lsz = padded_len(Q);
    const int wsh = g.twlg - (g.lgQ + 1);
    // Z_k = (X_k + conj X_{Q-k}) + i e^{2 pi i k / P1} (X_k - conj X_{Q-k}), k < Q
    auto src = [&](int l, int k) -> Cx<T> {
        const int L = l0 + l, row = L / 3, c = L - 3 * row;
        const Cx<T> *s = b.S + c * g.s_comp + ((long)(row / g.N2) * g.P2 + row % g.N2) * g.Xp;
        const Cx<T> Xk = s[k], Xc = conj(s[Q - k]);
        return (Xk + Xc) + mul_si((Xk - Xc) * conj(b.tw[k << wsh]), 1);
    };
    auto sm = [&](int l, int i) { return l * lsz + pad16(i); };
    auto dst = [&](int l, int j, Cx<T> v) {
        const int L = l0 + l, row = L / 3, c = L - 3 * row;
        const long cell = (long)row * g.N1 + 2 * j;  // row = zz * N2 + yy
        put(c, cell, v.x);
        if (2 * j + 1 < g.N1) put(c, cell + 1, v.y);
    };
    fft_lines<T, false, false, false>(buf, nl, g.lgQ, +1, b.tw, g.twlg, Q, (g.N1 + 1) >> 1, src, sm, dst);
}

// Passes 2 and 4: y transform of G consecutive kx columns of one (component, z) plane, in place.
// Forward reads y < N2 (zero padding above) and writes all P2; inverse reads all P2, writes y < N2.
// The rows are staged with cp.async (all in flight at once), the last stage writes global memory.
template <typename T>
__global__ void __launch_bounds__(512) k_y(Geom g, DemagBufs<T> b, int G, int dir)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *base = b.S + (long)blockIdx.y * g.P2 * g.Xp + blockIdx.x * G;
    const int nin = dir < 0 ? g.N2 : g.P2, nout = dir < 0 ? g.P2 : g.N2;
    const int Xp = g.Xp;
    const int rowb = G * (int)sizeof(Cx<T>);
    const int cb = rowb >= 16 ? 16 : rowb;  // bytes per async copy
    const int cpr = rowb / cb;
    for (int t = threadIdx.x; t < nin * cpr; t += blockDim.x) {
        const int y = t / cpr, ch = t - y * cpr;
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
    fft_lines<T, true, true, false>(buf, G, g.lgP2, dir, b.tw, g.twlg, nin, nout, sm_src, sm, dst);
}

// H^ = N~ M^ at one frequency; N~ real symmetric, stored on the octant with the odd components'
// signs restored here (Nxy odd in ky, Nxz odd in kz, Nyz odd in both).
template <typename T>
__device__ __forceinline__ void tensor_apply(const Geom &g, const DemagBufs<T> &b, int kx, int ky, int kz, Cx<T> &mx,
                                             Cx<T> &my, Cx<T> &mz)
{
    const int h2 = g.P2 >> 1, h3 = g.P3 >> 1;
    const int a2 = ky <= h2 ? ky : g.P2 - ky;
    const int a3 = kz <= h3 ? kz : g.P3 - kz;
    const T s2 = ky <= h2 ? T(1) : T(-1);
    const T s3 = kz <= h3 ? T(1) : T(-1);
    const T *n = b.Nk + ((long)a3 * g.H2 + a2) * g.Xp + kx;
    const long tc = g.t_comp;
    const T nxx = n[0], nyy = n[tc], nzz = n[2 * tc];
    const T nxy = n[3 * tc] * s2, nxz = n[4 * tc] * s3, nyz = n[5 * tc] * (s2 * s3);
    const Cx<T> hx = cx<T>(nxx * mx.x + nxy * my.x + nxz * mz.x, nxx * mx.y + nxy * my.y + nxz * mz.y);
    const Cx<T> hy = cx<T>(nxy * mx.x + nyy * my.x + nyz * mz.x, nxy * mx.y + nyy * my.y + nyz * mz.y);
    const Cx<T> hz = cx<T>(nxz * mx.x + nyz * my.x + nzz * mz.x, nxz * mx.y + nyz * my.y + nzz * mz.y);
    mx = hx; my = hy; mz = hz;
}

// Pass 3 (N3 > 1): for G kx columns and KY ky rows: forward z (N3 non-zero inputs), tensor product,
// inverse z keeping z < N3.  Lines l = (c * KY + kyl) * G + g, innermost in shared memory.
template <typename T>
__global__ void __launch_bounds__(512) k_z_conv(Geom g, DemagBufs<T> b, int G, int KY)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int kx0 = blockIdx.x * G, ky0 = blockIdx.y * KY;
    const int nl = 3 * KY * G;
    auto gaddr = [&](int l, int z) -> long {
        const int gg = l % G, r = l / G, kyl = r % KY, c = r / KY;
        return c * g.s_comp + ((long)z * g.P2 + ky0 + kyl) * g.Xp + kx0 + gg;
    };
    auto sm = [&](int l, int i) { return pad16(i) * nl + l; };
    auto sm_src = [&](int l, int i) { return buf[pad16(i) * nl + l]; };
    auto dst = [&](int l, int z, Cx<T> v) { b.S[gaddr(l, z)] = v; };
    {
        // rows (z, c, kyl) of G complex values, staged with cp.async
        const int rowb = G * (int)sizeof(Cx<T>);
        const int cb = rowb >= 16 ? 16 : rowb, cpr = rowb / cb;
        const int nrow = g.N3 * 3 * KY;
        for (int t = threadIdx.x; t < nrow * cpr; t += blockDim.x) {
            const int rr = t / cpr, ch = t - rr * cpr;
            const int kyl = rr % KY, c = (rr / KY) % 3, z = rr / (3 * KY);
            const int l = (c * KY + kyl) * G;
            char *d = (char *)(buf + pad16(z) * nl + l) + ch * cb;
            const char *s = (const char *)(b.S + gaddr(l, z)) + ch * cb;
            if (cb == 16) cp_async16(d, s);
            else cp_async8(d, s);
        }
        cp_async_wait_all();
        __syncthreads();
    }
    fft_lines<T, true, true, true>(buf, nl, g.lgP3, -1, b.tw, g.twlg, g.N3, g.P3, sm_src, sm, [&](int l, int i, Cx<T> v) { buf[pad16(i) * nl + l] = v; });
    const int npts = KY * G * g.P3;
    for (int t = threadIdx.x; t < npts; t += blockDim.x) {
        const int gg = t % G, r = t / G, kyl = r % KY, kz = r / KY;
        const int l0 = kyl * G + gg;
        Cx<T> *px = buf + pad16(kz) * nl + l0;
        Cx<T> *py = px + KY * G;
        Cx<T> *pz = py + KY * G;
        Cx<T> mx = *px, my = *py, mz = *pz;
        tensor_apply(g, b, kx0 + gg, ky0 + kyl, kz, mx, my, mz);
        *px = mx; *py = my; *pz = mz;
    }
    __syncthreads();
    fft_lines<T, true, true, false>(buf, nl, g.lgP3, +1, b.tw, g.twlg, g.P3, g.N3, sm_src, sm, dst);
}

// Single-layer variant (N3 == 1, P3 == 1): forward y, tensor product at kz = 0, inverse y.
// Lines l = c * G + g.
template <typename T>
__global__ void __launch_bounds__(512) k_y_conv(Geom g, DemagBufs<T> b, int G)
{
    if (b.ctl && b.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int kx0 = blockIdx.x * G;
    const int nl = 3 * G;
    auto gaddr = [&](int l, int y) -> long {
        const int gg = l % G, c = l / G;
        return c * g.s_comp + (long)y * g.Xp + kx0 + gg;
    };
    auto sm = [&](int l, int i) { return pad16(i) * nl + l; };
    auto sm_dst = [&](int l, int i, Cx<T> v) { buf[pad16(i) * nl + l] = v; };
    auto sm_src = [&](int l, int i) { return buf[pad16(i) * nl + l]; };
    auto dst = [&](int l, int y, Cx<T> v) { b.S[gaddr(l, y)] = v; };
    {
        const int rowb = G * (int)sizeof(Cx<T>);
        const int cb = rowb >= 16 ? 16 : rowb, cpr = rowb / cb;
        const int nrow = g.N2 * 3;
        for (int t = threadIdx.x; t < nrow * cpr; t += blockDim.x) {
            const int rr = t / cpr, ch = t - rr * cpr;
            const int c = rr % 3, y = rr / 3;
            char *d = (char *)(buf + pad16(y) * nl + c * G) + ch * cb;
            const char *s = (const char *)(b.S + gaddr(c * G, y)) + ch * cb;
            if (cb == 16) cp_async16(d, s);
            else cp_async8(d, s);
        }
        cp_async_wait_all();
        __syncthreads();
    }
    fft_lines<T, true, true, true>(buf, nl, g.lgP2, -1, b.tw, g.twlg, g.N2, g.P2, sm_src, sm, sm_dst);
    for (int t = threadIdx.x; t < G * g.P2; t += blockDim.x) {
        const int gg = t % G, ky = t / G;
        Cx<T> *px = buf + pad16(ky) * nl + gg;
        Cx<T> *py = px + G;
        Cx<T> *pz = py + G;
        Cx<T> mx = *px, my = *py, mz = *pz;
        tensor_apply(g, b, kx0 + gg, ky, 0, mx, my, mz);
        *px = mx; *py = my; *pz = mz;
    }
    __syncthreads();
    fft_lines<T, true, true, false>(buf, nl, g.lgP2, +1, b.tw, g.twlg, g.P2, g.N2, sm_src, sm, dst);
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

static int pow2_floor(int v)
{
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

// threads for a block transforming `elems` complex values (fft_regs<T>() per thread), 256 or 512
template <typename T>
static int threads_for(long elems)
{
    return elems > (long)fft_regs<T>() * 256 ? 512 : 256;
}

template <typename T>
DemagPlan demag_plan(const Geom &g)
{
    DemagPlan p{};
    p.ok = true;
    const size_t cs = sizeof(Cx<T>);
    const long kMaxElems = (long)fft_regs<T>() * 512;
    const int nlines = 3 * g.N2 * g.N3;
    {
        const int Q = g.P1 == 1 ? 1 : g.Q;
        int lpb = (int)(kMaxElems / Q);
        if (lpb < 1) p.ok = false;
        lpb = lpb < 1 ? 1 : lpb;
        lpb = lpb > 48 ? 48 : lpb;
        lpb = lpb > nlines ? nlines : lpb;
        p.x_lpb = lpb;
        p.x_threads = threads_for<T>((long)lpb * Q);
        p.x_smem = g.P1 == 1 ? 0 : (size_t)lpb * padded_len(Q) * cs;
    }
    if (g.N3 > 1) {
        int G = pow2_floor((int)(kMaxElems / g.P2));
        if ((long)G * g.P2 > kMaxElems) p.ok = false;
        G = G > 16 ? 16 : G;
        p.y_G = G;
        p.y_threads = threads_for<T>((long)G * g.P2);
        p.y_smem = (size_t)padded_len(g.P2) * G * cs;
        int Gz = pow2_floor((int)(kMaxElems / (3L * g.P3)));
        Gz = Gz > 16 ? 16 : Gz;
        if (3L * Gz * g.P3 > kMaxElems) p.ok = false;
        int KY = pow2_floor((int)(kMaxElems / (3L * Gz * g.P3)));
        KY = KY > g.P2 ? g.P2 : KY;
        p.z_G = Gz;
        p.z_KY = KY;
        p.z_threads = threads_for<T>(3L * KY * Gz * g.P3);
        p.z_smem = (size_t)padded_len(g.P3) * 3 * KY * Gz * cs;
    } else {
        int G = pow2_floor((int)(kMaxElems / (3L * g.P2)));
        if (3L * G * g.P2 > kMaxElems) p.ok = false;
        G = G > 16 ? 16 : G;
        p.yc_G = G;
        p.yc_threads = threads_for<T>(3L * G * g.P2);
        p.yc_smem = (size_t)padded_len(g.P2) * 3 * G * cs;
    }
    // every grid dimension divides Xp (a multiple of 16)
    if (g.Xp % (g.N3 > 1 ? (p.y_G > p.z_G ? p.y_G : p.z_G) : p.yc_G) != 0) p.ok = false;
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
        k_z_conv<T><<<dim3(g.Xp / p.z_G, div_up(g.P2, p.z_KY)), p.z_threads, p.z_smem, st>>>(g, b, p.z_G, p.z_KY);
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
