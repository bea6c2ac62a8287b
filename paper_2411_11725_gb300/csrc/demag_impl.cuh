// Demag passes (section "Demagnetization Field"): node->cell averaging fused into a pruned
// real-to-complex x transform, pruned y transforms, a z pass that fuses forward z, the pointwise
// product with the symmetric tensor spectrum and inverse z (or, for one cell layer, a y pass that
// fuses forward y, the product and inverse y), and a pruned complex-to-real x transform that writes
// Ms_c H_c per cell.
//
// Every kernel is instantiated per log2 transform length (the f3 engine), so the index arithmetic of
// the FFT stages is resolved at compile time.  The x passes read their input in the first FFT stage
// straight from global memory (the zero padding is never read); the forward y pass and the z passes
// stage their strided tiles in shared memory with cp.async (all copies of a tile in flight at once), the
// inverse y pass with one TMA tensor copy per tile, and the forward y pass writes its tile back with one
// TMA tensor store.  Every pass writes its
// output from the last FFT stage straight to global memory, and only the part that later passes read.
//
// Templates only: demag_f32.cu and demag_f64.cu instantiate them (two translation units, compiled in
// parallel).
#pragma once
#include <string.h>

#include "demag.cuh"
#include "fft3.cuh"

namespace nm {

// x passes: small blocks hide the gather and barrier latency best (measured against 256 and 512
// threads): the forward pass takes 128 threads (two 1024-point lines, eight blocks per SM), the inverse
// pass 64 in FP32 (one line, sixteen blocks per SM; FP64 keeps 128 threads for its 8 values per thread)
constexpr int kXThreads = 128;
template <typename T>
constexpr int kXiThreads = sizeof(T) == 4 ? 64 : 128;
// y and z passes: 512-thread blocks, two per SM in FP32 (one block's loads and barriers overlap the
// other's arithmetic); the longest y lines (2^11) take 1024 threads so that a block still spans 4 columns.
template <typename T, int LG = 0>
constexpr int kMaxThreads = 512;
template <typename T, int LG = 0>
constexpr int kMinBlocks = sizeof(T) == 4 ? 2 : 1;
// values per thread per FFT stage in the y passes: radix-16 stages for the long FP32 lines
template <typename T, int LG>
constexpr int kYEpt = (sizeof(T) == 4 && LG >= 10) ? 16 : 8;
constexpr int pow2_floor_c(int v)
{
    int p = 1;
    while (2 * p <= v) p *= 2;
    return p;
}
// Compile-time tile of the z convolution for lines of 2^LG: G kx columns x KY octant rows (each with its
// mirror) x 3 components, 16 values per thread for short FP32 lines (128-byte rows), 8 otherwise.
template <typename T, int LG>
struct ZTile {
    static constexpr int P3 = 1 << LG;
    static constexpr int EPT = (sizeof(T) == 4 && LG <= 5) ? 16 : 8;
    static constexpr int BUDGET = EPT * kMaxThreads<T>;
    static constexpr int G0 = EPT == 16 ? 16 : (int)(64 / sizeof(Cx<T>));
    static constexpr int fit_g(int g) { return (g > 1 && 6 * g * P3 > BUDGET) ? fit_g(g / 2) : g; }
    static constexpr int G = fit_g(G0);
    static constexpr int KY = pow2_floor_c(BUDGET / (6 * G * P3)) > 0 ? pow2_floor_c(BUDGET / (6 * G * P3)) : 1;
    static constexpr int NL = 6 * KY * G;
    static constexpr int THREADS = ((NL * P3 / EPT > 32 ? NL * P3 / EPT : 32) + 31) / 32 * 32;
    static constexpr size_t SMEM = (size_t)NL * P3 * sizeof(Cx<T>) + (size_t)6 * (P3 / 2 + 1) * KY * G * sizeof(T);
    static_assert(NL * P3 <= EPT * THREADS && THREADS <= kMaxThreads<T>, "z tile exceeds the block");
};

// Compile-time tile of the y passes for lines of 2^LG: G kx columns, EPT values per thread.  Tiles of
// fewer than 16 columns pad the lines-fastest layout with one row every 8 elements (LFP = 3): the first
// stage stores with a stride of radix x G elements, which otherwise hits the same banks.
template <typename T, int LG>
struct YTile {
    static constexpr int P2 = 1 << LG;
    static constexpr int EPT = kYEpt<T, LG>;
    static constexpr int MAXT = kMaxThreads<T, LG>;
    static constexpr int G0 = pow2_floor_c(EPT * MAXT / P2);
    static constexpr int G = G0 > 16 ? 16 : (G0 < 1 ? 1 : G0);
    static constexpr int LFP = G < 16 ? 3 : 0;
    static constexpr int THREADS = ((G * P2 / EPT > 32 ? G * P2 / EPT : 32) + 31) / 32 * 32;
    static constexpr size_t SMEM = (size_t)G * f3::lf_rows(P2, LFP) * sizeof(Cx<T>), TILE_BYTES = SMEM;
    // inverse pass: the tile, up to 128 bytes to align it for the TMA copy, and the copy's barrier
    static constexpr size_t SMEM_TMA = TILE_BYTES + 128 + 16;
    static_assert(G * P2 <= EPT * THREADS && THREADS <= MAXT, "y tile exceeds the block");
    static_assert(TILE_BYTES % 8 == 0, "barrier alignment");
};

// x passes: radix-16 stages for FP32 lines of 2^10 complex values
template <typename T, int LG>
constexpr int kXEpt = (sizeof(T) == 4 && LG >= 10) ? 16 : 8;
// the single-layer pass keeps up to 1024 threads (FP32) so that long y lines still fit one block
template <typename T>
constexpr int kMaxThreadsYC = sizeof(T) == 4 ? 1024 : 512;

// Asynchronous global -> shared copies (cp.async): many in flight per thread without registers.
__device__ __forceinline__ void cpa16(void *sm, const void *gm)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(sm)),
                 "l"(gm)
                 : "memory");
}
__device__ __forceinline__ void cpa8(void *sm, const void *gm)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(sm)),
                 "l"(gm)
                 : "memory");
}
__device__ __forceinline__ void cpa_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
// copy `bytes` (a multiple of 8; both addresses aligned to min(bytes, 16)) as copy number ch of a row
__device__ __forceinline__ void cpa_chunk(void *sm, const void *gm, int cb)
{
    if (cb == 16) cpa16(sm, gm);
    else cpa8(sm, gm);
}

// x-pass line L = c * (N2 N3) + row, row = zz * N2 + yy: consecutive lines of a block are consecutive
// cell rows of one component, so the node rows they average overlap.  Offsets (elements, int32: every
// supported size fits) of the line's start in the node array, the cell arrays and the spectrum.
struct XInfo {
    int in;    // node array (nodal input) or cell array (cell input / output), component included
    int cell;  // cell index of the row start (Ms map)
    int spec;  // spectrum row start
};
__device__ __forceinline__ XInfo x_info(const Geom &g, const FastDiv &nrf, int L, bool cell_in)
{
    const int NR = g.N2 * g.N3;
    const int c = (int)nrf.div((unsigned)L);
    const int row = L - c * NR;
    const int zz = (int)g.n2f.div((unsigned)row);
    const int yy = row - zz * g.N2;
    XInfo x;
    x.cell = row * g.N1;
    x.in = cell_in ? c * (int)g.cs + x.cell : c * (int)g.ns + zz * g.zsn + yy * g.ysn;
    x.spec = c * (int)g.s_comp + (zz * g.P2 + yy) * g.Xp;
    return x;
}

// M of the cell pair (x, x+1) of a row: M_c = Ms_c * (1/8) sum_{i in {0,1}^3} y_{c+i}.  p points at node
// (x, yy, zz) of one component; `row` is the node offset of the upper y corners (0 with the 1D basis) and
// `plane` that of the upper z corners (0 with the 2D and 1D bases, where the 8-corner mean is the mean of
// the 4 in-plane corners, or of the 2 corners along x).
template <typename T>
__device__ __forceinline__ Cx<T> cell_M_pair(const T *__restrict__ p, int row, int plane, const T *__restrict__ Ms,
                                             T Ms0, int cell, bool has2)
{
    const T a0 = (p[0] + p[row]) + (p[plane] + p[plane + row]);
    const T a1 = (p[1] + p[row + 1]) + (p[plane + 1] + p[plane + row + 1]);
    const T ms0 = Ms ? Ms[cell] : Ms0;
    T m0 = ms0 * T(0.125) * (a0 + a1), m1 = T(0);
    if (has2) {
        const T a2 = (p[2] + p[row + 2]) + (p[plane + 2] + p[plane + row + 2]);
        const T ms1 = Ms ? Ms[cell + 1] : Ms0;
        m1 = ms1 * T(0.125) * (a1 + a2);
    }
    return cx<T>(m0, m1);
}

// Pass 1: x transform (R2C of length P1 = 2Q via a complex FFT of length Q = 2^LG on even/odd pairs).
// One block holds `lpb` consecutive lines.  CELL_IN: the input is already a cell field.
template <typename T, bool CELL_IN, int LG>
__global__ void __launch_bounds__(kXThreads, sizeof(T) == 4 ? 8 : 4)
    k_x_fwd(Geom g, DemagBufs<T> b, const T *__restrict__ in, int lpb)
{
    if (b.ctl && b.ctl->done) return;
    constexpr int Q = 1 << LG, H = Q / 2, LSZ = f3::padded(Q);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    XInfo *info = reinterpret_cast<XInfo *>(buf + lpb * LSZ);
    const int nlines = 3 * g.N2 * g.N3;
    const int l0 = blockIdx.x * lpb;
    const int nl = min(lpb, nlines - l0);
    if (nl <= 0) return;
    if (threadIdx.x < nl) info[threadIdx.x] = x_info(g, FastDiv((unsigned)(g.N2 * g.N3)), l0 + threadIdx.x, CELL_IN);
    __syncthreads();
    const int N1 = g.N1, row = g.ysn, plane = g.zsn;  // 2D (1D) basis: both z (y and z) corners are the node
    const T *Ms = b.Ms;
    const T Ms0 = b.Ms0;
    auto src = [&](int l, int i) -> Cx<T> {
        const int x = 2 * i;
        const XInfo xi = info[l];
        const T *p = in + xi.in + x;
        if (CELL_IN) return cx<T>(p[0], x + 1 < N1 ? p[1] : T(0));
        return cell_M_pair<T>(p, row, plane, Ms, Ms0, xi.cell + x, x + 1 < N1);
    };
    f3::fft<T, LG, -1, false, false, true, kXEpt<T, LG>>(buf, nl, FastDiv(1u), b.tw, g.twlg, (N1 + 1) >> 1, Q, src,
                                                         f3::NoFn<T>());
    // X_k = (Z_k + conj Z_{Q-k})/2 - (i/2) W^k (Z_k - conj Z_{Q-k}),  W = e^{-2 pi i / P1},  k = 0..Q;
    // thread (l, k) with k < Q/2 writes X_k and X_{Q-k}; k = 0 also writes X_{Q/2} (and X_0, X_Q)
    const int wsh = g.twlg - (LG + 1);
    const Cx<T> *tw = b.tw;
    auto xk = [&](Cx<T> Zk, Cx<T> Zq, int k) -> Cx<T> {
        const Cx<T> Zc = conj(Zq);
        const Cx<T> E = scale(Zk + Zc, T(0.5));
        const Cx<T> O = scale(mul_si(Zk - Zc, -1), T(0.5));
        return E + tw[k << wsh] * O;
    };
    for (int t = threadIdx.x; t < nl * H; t += blockDim.x) {
        const int l = t >> (LG - 1 < 0 ? 0 : LG - 1), k = t & (H - 1);
        const Cx<T> *z = buf + l * LSZ;
        Cx<T> *out = b.S + info[l].spec;
        if (k == 0) {
            const Cx<T> Z0 = z[0];
            out[0] = xk(Z0, Z0, 0);
            out[Q] = xk(Z0, Z0, Q);
            if (H > 0 && Q > 1) {
                const Cx<T> Zh = z[f3::pad16c(H)];
                out[H] = xk(Zh, Zh, H);
            }
        } else {
            const Cx<T> Zk = z[f3::pad16c(k)], Zq = z[f3::pad16c(Q - k)];
            out[k] = xk(Zk, Zq, k);
            out[Q - k] = xk(Zq, Zk, Q - k);
        }
    }
}

// N1 == 1 (P1 == 1): the x "transform" is a copy of the cell value (real) into kx = 0.
template <typename T, bool CELL_IN>
__global__ void k_x_fwd1(Geom g, DemagBufs<T> b, const T *__restrict__ in)
{
    if (b.ctl && b.ctl->done) return;
    const int nlines = 3 * g.N2 * g.N3;
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= nlines) return;
    const XInfo xi = x_info(g, FastDiv((unsigned)(g.N2 * g.N3)), L, CELL_IN);
    T v;
    if (CELL_IN) v = in[xi.in];
    else v = cell_M_pair<T>(in + xi.in, g.ysn, g.zsn, b.Ms, b.Ms0, xi.cell, false).x;
    b.S[xi.spec] = cx<T>(v, T(0));
}

// Pass 5: inverse x transform (C2R of length P1 via a complex FFT of length Q), keeping x < N1.
// Output per cell: Ms_c H_c (or H_c when CELL_OUT).
template <typename T, bool CELL_OUT, int LG>
__global__ void __launch_bounds__(kXiThreads<T>, sizeof(T) == 4 ? 16 : 4)
    k_x_inv(Geom g, DemagBufs<T> b, T *__restrict__ out, int lpb)
{
    if (b.ctl && b.ctl->done) return;
    constexpr int Q = 1 << LG, H = Q / 2, LSZ = f3::padded(Q);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    XInfo *info = reinterpret_cast<XInfo *>(buf + lpb * LSZ);
    const int nlines = 3 * g.N2 * g.N3;
    const int l0 = blockIdx.x * lpb;
    const int nl = min(lpb, nlines - l0);
    if (nl <= 0) return;
    if (threadIdx.x < nl) info[threadIdx.x] = x_info(g, FastDiv((unsigned)(g.N2 * g.N3)), l0 + threadIdx.x, true);
    __syncthreads();
    // Z_k = (X_k + conj X_{Q-k}) + i conj(W^k) (X_k - conj X_{Q-k}), k < Q, into shared memory
    const int wsh = g.twlg - (LG + 1);
    const Cx<T> *tw = b.tw;
    auto zk = [&](Cx<T> Xk, Cx<T> Xq, int k) -> Cx<T> {
        const Cx<T> Xc = conj(Xq);
        return (Xk + Xc) + mul_si((Xk - Xc) * conj(tw[k << wsh]), 1);
    };
    // the spectrum reads of KB pairs per thread are issued together, before any of them is used
    constexpr int KB = 8;
    for (int t0 = threadIdx.x; t0 < nl * H; t0 += KB * blockDim.x) {
        Cx<T> xa[KB], xb[KB];
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int t = t0 + u * blockDim.x;
            if (t >= nl * H) break;
            const int l = t >> (LG - 1 < 0 ? 0 : LG - 1), k = t & (H - 1);
            const Cx<T> *s = b.S + info[l].spec;
            xa[u] = s[k];
            xb[u] = s[k == 0 ? Q : Q - k];
        }
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int t = t0 + u * blockDim.x;
            if (t >= nl * H) break;
            const int l = t >> (LG - 1 < 0 ? 0 : LG - 1), k = t & (H - 1);
            Cx<T> *z = buf + l * LSZ;
            if (k == 0) {
                z[0] = zk(xa[u], xb[u], 0);
                if (H > 0 && Q > 1) {
                    const Cx<T> Xh = b.S[info[l].spec + H];
                    z[f3::pad16c(H)] = zk(Xh, Xh, H);
                }
            } else {
                z[f3::pad16c(k)] = zk(xa[u], xb[u], k);
                z[f3::pad16c(Q - k)] = zk(xb[u], xa[u], Q - k);
            }
        }
    }
    __syncthreads();
    const int N1 = g.N1;
    const T *Ms = b.Ms;
    const T Ms0 = b.Ms0;
    auto dst = [&](int l, int j, Cx<T> v) {
        const XInfo xi = info[l];
        const int x = 2 * j;
        T v0 = v.x, v1 = v.y;
        if (!CELL_OUT) {
            v0 *= Ms ? Ms[xi.cell + x] : Ms0;
            if (x + 1 < N1) v1 *= Ms ? Ms[xi.cell + x + 1] : Ms0;
        }
        out[xi.in + x] = v0;
        if (x + 1 < N1) out[xi.in + x + 1] = v1;
    };
    f3::fft<T, LG, +1, false, true, false, kXEpt<T, LG>>(buf, nl, FastDiv(1u), b.tw, g.twlg, Q, (N1 + 1) >> 1, f3::NoFn<T>(), dst);
}

template <typename T, bool CELL_OUT>
__global__ void k_x_inv1(Geom g, DemagBufs<T> b, T *__restrict__ out)
{
    if (b.ctl && b.ctl->done) return;
    const int nlines = 3 * g.N2 * g.N3;
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= nlines) return;
    const XInfo xi = x_info(g, FastDiv((unsigned)(g.N2 * g.N3)), L, true);
    T v = b.S[xi.spec].x;
    if (!CELL_OUT) v *= b.Ms ? b.Ms[xi.cell] : b.Ms0;
    out[xi.in] = v;
}

// Shared-memory barriers and TMA tile copies (cp.async.bulk.tensor): one thread issues the copy of a
// block's whole tile, which completes on an mbarrier with its byte count; the threads wait on the
// barrier's phase.  Every wait is bounded (about a second of SM clock): a wait that runs out reports
// NM_ERR_TIMEOUT through the status word and the block writes nothing.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity)
{
    const long long t0 = clock64();
    for (unsigned it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > (2LL << 30)) break;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *tm, int c0, int c1, int c2, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"((unsigned long long)tm), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3,
                                            unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(dst),
        "l"((unsigned long long)tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// TMA tile store from shared memory (bulk group); the writes of the threads that filled the tile must
// be made visible to the copy first (fence_proxy_async by every writer, then a barrier)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *tm, int c0, int c1, int c2, unsigned src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
                     (unsigned long long)tm),
                 "r"(c0), "r"(c1), "r"(c2), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *tm, int c0, int c1, int c2, int c3, unsigned src)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n" ::"l"(
                     (unsigned long long)tm),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
                 : "memory");
}
// commit the issued stores and wait until they have read their shared-memory source
__device__ __forceinline__ void tma_store_commit_wait_read()
{
    asm volatile("cp.async.bulk.commit_group;\ncp.async.bulk.wait_group.read 0;\n" ::: "memory");
}

// Bytes of the inverse y pass's TMA tile copy (all P2 rows): groups of 8 rows plus the zero-filled
// padding row when the tile pads its rows (LFP = 3), plain rows otherwise (the box of demag_encode_ymap)
template <typename T, int LG>
__host__ __device__ constexpr unsigned y_tile_bytes()
{
    constexpr unsigned rowb = YTile<T, LG>::G * (unsigned)sizeof(Cx<T>), rows = 1u << LG;
    return YTile<T, LG>::LFP > 0 ? rows / 8 * 9u * rowb : rows * rowb;
}

// Passes 2 and 4: y transform of G consecutive kx columns of one (component, z) plane, in place.
// Forward reads y < N2 (zero padding above) and writes all P2; inverse reads all P2, writes y < N2.
// Shared layout: row y at buf + lfpad(y) * G (lines = columns, fastest; padded rows for narrow tiles).
//
// Forward y pass: the N2 input rows of the tile are staged with cp.async (all copies in flight at once;
// a TMA copy of the same rows measured slower here, 0.693 against 0.674 ms at 1024x1024x32).  The last
// stage writes the P2 outputs back into the tile, and one TMA store writes the whole tile (the box of
// the inverse pass's load, descriptor tm: its ninth row per group of 8 lies outside the tensor and is
// not written): 0.588 against 0.674 ms with the last stage storing to global memory itself.
template <typename T, int LG>
__global__ void __launch_bounds__(kMaxThreads<T, LG>, kMinBlocks<T, LG>)
    k_y_fwd(Geom g, DemagBufs<T> b, const __grid_constant__ CUtensorMap tm)
{
    if (b.ctl && b.ctl->done) return;
    constexpr int P2 = 1 << LG, G = YTile<T, LG>::G, LFP = YTile<T, LG>::LFP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the tile at the first 128-byte boundary of the dynamic buffer (the source of the TMA store)
    const unsigned pad = (128u - (smem_u32(smem_raw) & 127u)) & 127u;
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw + pad);
    const Cx<T> *base = b.S + (long)blockIdx.y * P2 * g.Xp + blockIdx.x * G;
    const int nin = g.N2;
    const int Xp = g.Xp;
    constexpr int rowb = G * (int)sizeof(Cx<T>);
    constexpr int cb = rowb >= 16 ? 16 : rowb;
    constexpr int cpr = rowb / cb;  // copies per row
    for (int t = threadIdx.x; t < nin * cpr; t += blockDim.x) {
        const int y = t / cpr, ch = t - y * cpr;
        cpa_chunk((char *)(buf + f3::lfpad<LFP>(y) * G) + ch * cb, (const char *)(base + y * Xp) + ch * cb, cb);
    }
    cpa_wait_all();
    __syncthreads();
    f3::fft<T, LG, -1, true, true, true, kYEpt<T, LG>, G, LFP>(buf, G, FastDiv(1u), b.tw, g.twlg, nin, P2,
                                                               f3::NoFn<T>(), f3::NoFn<T>());
    fence_proxy_async();  // (the transform ends with a barrier; this one orders the copy after every fence)
    __syncthreads();
    if (threadIdx.x == 0) {
        const int x0 = 2 * G * blockIdx.x;  // real elements: a multiple of 2G, i.e. of 16 bytes
        if constexpr (LFP > 0) tma_store_4d(&tm, x0, 0, 0, blockIdx.y, smem_u32(buf));
        else tma_store_3d(&tm, x0, 0, blockIdx.y, smem_u32(buf));
        tma_store_commit_wait_read();
    }
}

// Inverse y pass: the whole P2-row tile arrives by one TMA copy (descriptor tm, built by
// demag_encode_ymap) that completes on a shared-memory barrier.  With padded rows the copy's box spans
// 9 rows of each group of 8, the ninth outside the tensor and zero-filled by the copy, so the box lands
// in the padded layout as it is.  0.610 against 0.658 ms with cp.async staging at 1024x1024x32.
template <typename T, int LG>
__global__ void __launch_bounds__(kMaxThreads<T, LG>, kMinBlocks<T, LG>)
    k_y_inv(Geom g, DemagBufs<T> b, const __grid_constant__ CUtensorMap tm)
{
    if (b.ctl && b.ctl->done) return;
    constexpr int G = YTile<T, LG>::G, LFP = YTile<T, LG>::LFP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the tile at the first 128-byte boundary of the dynamic buffer, the barrier behind it
    const unsigned pad = (128u - (smem_u32(smem_raw) & 127u)) & 127u;
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw + pad);
    const unsigned bar = smem_u32(smem_raw + pad + YTile<T, LG>::TILE_BYTES);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, y_tile_bytes<T, LG>());
        const int x0 = 2 * G * blockIdx.x;  // real elements: a multiple of 2G, i.e. of 16 bytes
        if constexpr (LFP > 0) tma_load_4d(smem_u32(buf), &tm, x0, 0, 0, blockIdx.y, bar);
        else tma_load_3d(smem_u32(buf), &tm, x0, 0, blockIdx.y, bar);
    }
    const bool arrived = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!arrived)) {
        if (threadIdx.x == 0 && b.wait_err) atomicExch(b.wait_err, NM_ERR_TIMEOUT);
        mbar_wait_bounded(bar, 0);  // the copy may still land: let it finish before the block exits
        return;
    }
    constexpr int P2 = 1 << LG;
    Cx<T> *base = b.S + (long)blockIdx.y * P2 * g.Xp + blockIdx.x * G;
    const int Xp = g.Xp;
    auto dst = [&](int l, int i, Cx<T> v) { base[i * Xp + l] = v; };
    f3::fft<T, LG, +1, true, true, false, kYEpt<T, LG>, G, LFP>(buf, G, FastDiv(1u), b.tw, g.twlg, P2, g.N2,
                                                                f3::NoFn<T>(), dst);
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

// ky of row r of a z tile whose octant rows start at a20: rows r < KY are ky = a20 + r, rows KY + r are
// the mirrors P2 - (a20 + r), present when 0 < a2 < P2/2; -1 marks an absent row
template <int KY>
__device__ __forceinline__ int z_row_ky(const Geom &g, int a20, int r)
{
    const int a2 = a20 + (r < KY ? r : r - KY);
    if (a2 >= g.H2) return -1;
    if (r < KY) return a2;
    return (a2 > 0 && a2 < (g.P2 >> 1)) ? g.P2 - a2 : -1;
}

// Stage a z tile in shared memory with cp.async: the N3 spectrum rows of its 3 x 2KY lines of G kx
// columns (element z of line l = (c * 2KY + r) * G + g at buf[z * nl + l]), then the tensor slice
// [component][a3][row][kx] behind the NL * P3 spectrum values; ends with a barrier.
template <typename T, int G, int KY, int P3, bool TENSOR = true>
__device__ __forceinline__ void z_tile_load(const Geom &g, const DemagBufs<T> &b, Cx<T> *buf, int kx0, int a20)
{
    constexpr int R2 = 2 * KY, nl = 3 * R2 * G, H3 = P3 / 2 + 1;
    constexpr int rowb = G * (int)sizeof(Cx<T>);
    constexpr int cb = rowb >= 16 ? 16 : rowb, lcpr = rowb / cb == 1 ? 0 : (rowb / cb == 2 ? 1 : (rowb / cb == 4 ? 2 : 3));
    const int nrow = g.N3 * 3 * R2;
    for (int t = threadIdx.x; t < (nrow << lcpr); t += blockDim.x) {
        const int rr = t >> lcpr, ch = t - (rr << lcpr);
        const int r = rr % R2, cz = rr / R2, z = cz / 3, c = cz - 3 * z;
        const int ky = z_row_ky<KY>(g, a20, r);
        if (ky < 0) continue;
        const long ga = c * g.s_comp + ((long)z * g.P2 + ky) * g.Xp + kx0;
        cpa_chunk((char *)(buf + z * nl + (c * R2 + r) * G) + ch * cb, (const char *)(b.S + ga) + ch * cb, cb);
    }
    // the tensor slice of this tile, copied while the spectrum rows arrive
    T *ten = reinterpret_cast<T *>(buf + nl * P3);
    constexpr int trowb = G * (int)sizeof(T);
    constexpr int tcb = trowb >= 16 ? 16 : trowb, tch = trowb / tcb;
    for (int t = threadIdx.x; TENSOR && t < 6 * H3 * KY * tch; t += blockDim.x) {
        const int row = t / tch, ch = t - row * tch;
        const int rr = row % KY, kq = row / KY, a3 = kq % H3, comp = kq / H3;
        const int a2 = a20 + rr;
        if (a2 >= g.H2) continue;
        cpa_chunk((char *)(ten + row * G) + ch * tcb,
                  (const char *)(b.Nk + comp * g.t_comp + ((long)a3 * g.H2 + a2) * g.Xp + kx0) + ch * tcb, tcb);
    }
    cpa_wait_all();
    __syncthreads();
}

// Pass 3 (N3 > 1): G kx columns x KY octant rows a2 (each with its mirror P2 - a2, so the tensor is
// read once): forward z (N3 non-zero inputs), tensor product, inverse z keeping z < N3.
// Rows r < KY are ky = a2_0 + r, rows KY + r are ky = P2 - (a2_0 + r) (present when 0 < a2 < P2/2).
// Lines l = (c * 2KY + r) * G + g; element kz of line l at buf[kz * nl + l].
template <typename T, int LG>
__global__ void __launch_bounds__(kMaxThreads<T>, kMinBlocks<T>) k_z_conv(Geom g, DemagBufs<T> b)
{
    if (b.ctl && b.ctl->done) return;
    using Z = ZTile<T, LG>;
    constexpr int P3 = 1 << LG, H3 = P3 / 2 + 1, G = Z::G, KY = Z::KY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int kx0 = blockIdx.x * G, a20 = blockIdx.y * KY;
    constexpr int R2 = 2 * KY, nl = 3 * R2 * G;
    const int h2 = g.P2 >> 1;
    auto row_ky = [&](int r) -> int { return z_row_ky<KY>(g, a20, r); };
    auto gaddr = [&](int c, int ky, int z) -> long { return c * g.s_comp + ((long)z * g.P2 + ky) * g.Xp + kx0; };
    z_tile_load<T, G, KY, P3>(g, b, buf, kx0, a20);
    const FastDiv nlf(1u);  // unused: the line count is a compile-time constant
    f3::fft<T, LG, -1, true, true, true, Z::EPT, nl>(buf, nl, nlf, b.tw, g.twlg, g.N3, P3, f3::NoFn<T>(),
                                                    f3::NoFn<T>());
    constexpr int npts = KY * G * P3;
    const T *ten = reinterpret_cast<const T *>(buf + nl * P3);
    constexpr int tstride = H3 * KY * G;
    for (int t = threadIdx.x; t < npts; t += blockDim.x) {
        const int gg = t % G, q = t / G, rr = q % KY, kz = q / KY;
        const int a2 = a20 + rr;
        if (a2 >= g.H2) continue;
        const int a3 = kz <= (P3 >> 1) ? kz : P3 - kz;
        const T s3 = kz <= (P3 >> 1) ? T(1) : T(-1);
        const T *tp = ten + (a3 * KY + rr) * G + gg;
        Ten6<T> tt;
        tt.xx = tp[0];
        tt.yy = tp[tstride];
        tt.zz = tp[2 * tstride];
        tt.xy = tp[3 * tstride];
        tt.xz = tp[4 * tstride] * s3;
        tt.yz = tp[5 * tstride] * s3;
        const Ten6<T> &ten6 = tt;
        Cx<T> *p = buf + kz * nl + rr * G + gg;
        tensor_mul(ten6, T(1), p, p + R2 * G, p + 2 * R2 * G);
        if (a2 > 0 && a2 < h2) {
            Cx<T> *pm = p + KY * G;
            tensor_mul(ten6, T(-1), pm, pm + R2 * G, pm + 2 * R2 * G);
        }
    }
    __syncthreads();
    auto dst = [&](int l, int z, Cx<T> v) {
        const int gg = l % G, q = l / G, r = q % R2, c = q / R2;
        const int ky = row_ky(r);
        if (ky >= 0) b.S[gaddr(c, ky, z) + gg] = v;
    };
    f3::fft<T, LG, +1, true, true, false, Z::EPT, nl>(buf, nl, nlf, b.tw, g.twlg, P3, g.N3, f3::NoFn<T>(), dst);
}

// Register z convolution (FP32, P3 = 2^LG <= 64).  The z input is zero above N3 <= P3/2, so with
// S threads per line (S = 2 or 4) and D = P3/S the spectrum splits into S interleaved parts:
//   X_{Sk+r} = sum_{m<D} e^{-2 pi i mk/D} w^{mr} sum_{j<S/2} w_S^{jr} x_{m+jD},
// w = e^{-2 pi i/P3}, w_S = w^D, and the inverse kept for z = m + jD < N3 is
//   y_{m+jD} = sum_r conj(w_S)^{jr} conj(w)^{mr} u_r[m],   u_r = length-D inverse transform of part r.
// Thread r of a line forms its part and runs the whole length-D transform in registers: no
// shared-memory exchange between FFT stages.  Shared layout: the tile of z_tile_load; after the forward
// transform, kz = Sk + r of line l sits in row rD + k; the inverse leaves conj(w)^{mr} u_r[m] in the same
// rows and the S threads of a line then share the sums over r.
template <int LG, int S>
struct ZRTile {
    static constexpr int P3 = 1 << LG, D = P3 / S, G = 16;
    static constexpr int KY0 = pow2_floor_c(56 * 1024 / (6 * G * P3 * 8));
    static constexpr int KY = KY0 < 1 ? 1 : (KY0 > 2 ? 2 : KY0);
    static constexpr int NL = 6 * KY * G;  // lines (a multiple of 32: warps hold one part r)
    static constexpr int THREADS = S * NL;
    // the tensor slice goes through shared memory, except for 64-point lines: there the product reads it
    // from global memory (L2), so that four blocks fit an SM
    static constexpr bool TSM = LG < 6;
    static constexpr size_t SMEM =
        (size_t)NL * P3 * sizeof(Cx<float>) + (TSM ? (size_t)6 * (P3 / 2 + 1) * KY * G * sizeof(float) : 0);
    static_assert(LG >= 2 && LG <= 6 && (S == 2 || S == 4) && D >= 2 && NL % 32 == 0 && THREADS <= 1024,
                  "register z tile");
};
// threads per line of the register z convolution: 2 (measured on 64-point lines: 1.21 ms against 1.59 ms
// with 4 threads of 16-point transforms, although those fit twice the resident warps)
template <int LG>
constexpr int kZRSplit = 2;

template <int LG>
__global__ void __launch_bounds__(ZRTile<LG, kZRSplit<LG>>::THREADS, kZRSplit<LG> == 4 ? 3 : (LG >= 6 ? 4 : 2))
    k_z_conv_r(Geom g, DemagBufs<float> b)
{
    using T = float;
    constexpr int S = kZRSplit<LG>;
    using Z = ZRTile<LG, S>;
    if (b.ctl && b.ctl->done) return;
    constexpr int P3 = Z::P3, D = Z::D, H = P3 / 2, H3 = H + 1, G = Z::G, KY = Z::KY, R2 = 2 * KY, nl = Z::NL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int kx0 = blockIdx.x * G, a20 = blockIdx.y * KY;
    z_tile_load<T, G, KY, P3, Z::TSM>(g, b, buf, kx0, a20);
    const int r = threadIdx.x / nl, l = threadIdx.x - r * nl;
    const int N3 = g.N3;
    {
        // forward: part r of the line's spectrum
        Cx<T> v[D];
#pragma unroll
        for (int m = 0; m < D; ++m) {
            v[m] = m < N3 ? buf[m * nl + l] : cx<T>(T(0), T(0));
            if (S == 4) {
                // x_{m+D} w_S^r, w_S = -i (forward)
                const Cx<T> x1 = m + D < N3 ? buf[(m + D) * nl + l] : cx<T>(T(0), T(0));
                const Cx<T> t = r == 0 ? x1 : (r == 1 ? mul_si(x1, -1) : (r == 2 ? cx<T>(-x1.x, -x1.y) : mul_si(x1, 1)));
                v[m] = f3::csum(v[m], t);
            }
        }
        __syncthreads();  // every part has read the input rows before any overwrites them
        if (r > 0) {
#pragma unroll
            for (int m = 1; m < D; ++m) {
                // w^{mr}: r is warp-uniform, the twiddle a compile-time constant per branch
                if (r == 1) v[m] = f3::rot<T, P3, -1>(v[m], m);
                else if (S == 4 && r == 2) v[m] = f3::rot<T, P3, -1>(v[m], 2 * m);
                else if (S == 4 && r == 3) v[m] = f3::rot<T, P3, -1>(v[m], 3 * m);
            }
        }
        f3::dft_reg<T, D, -1>(v);
#pragma unroll
        for (int k = 0; k < D; ++k) buf[(r * D + k) * nl + l] = v[f3::bitrev<D>(k)];
    }
    __syncthreads();
    {
        // H^ = N~ M^ at every (kz, row, kx) of the tile; row q holds kz = S (q mod D) + q / D
        const T *ten = reinterpret_cast<const T *>(buf + nl * P3);
        constexpr int tstride = H3 * KY * G, npts = KY * G * P3;
        const int h2 = g.P2 >> 1;
        if constexpr (!Z::TSM) {
            // the tensor comes from L2: all of a thread's tensor reads are issued before the products
            constexpr int NPT = (npts + Z::THREADS - 1) / Z::THREADS;
            Ten6<T> tv[NPT];
#pragma unroll
            for (int u = 0; u < NPT; ++u) {
                const int t = threadIdx.x + u * Z::THREADS;
                const int gg = t % G, qr = t / G, rr = qr % KY, q = qr / KY;
                const int a2 = a20 + rr;
                if (t >= npts || a2 >= g.H2) continue;
                const int kz = S * (q % D) + q / D;
                const int a3 = kz <= H ? kz : P3 - kz;
                const T *tp = b.Nk + ((long)a3 * g.H2 + a2) * g.Xp + kx0 + gg;
                const long tc = g.t_comp;
                tv[u].xx = __ldg(tp);
                tv[u].yy = __ldg(tp + tc);
                tv[u].zz = __ldg(tp + 2 * tc);
                tv[u].xy = __ldg(tp + 3 * tc);
                tv[u].xz = __ldg(tp + 4 * tc);
                tv[u].yz = __ldg(tp + 5 * tc);
            }
#pragma unroll
            for (int u = 0; u < NPT; ++u) {
                const int t = threadIdx.x + u * Z::THREADS;
                const int gg = t % G, qr = t / G, rr = qr % KY, q = qr / KY;
                const int a2 = a20 + rr;
                if (t >= npts || a2 >= g.H2) continue;
                const int kz = S * (q % D) + q / D;
                const T s3 = kz <= H ? T(1) : T(-1);
                Ten6<T> tt = tv[u];
                tt.xz *= s3;
                tt.yz *= s3;
                Cx<T> *p = buf + q * nl + rr * G + gg;
                tensor_mul(tt, T(1), p, p + R2 * G, p + 2 * R2 * G);
                if (a2 > 0 && a2 < h2) {
                    Cx<T> *pm = p + KY * G;
                    tensor_mul(tt, T(-1), pm, pm + R2 * G, pm + 2 * R2 * G);
                }
            }
        }
#pragma unroll 2
        for (int t = threadIdx.x; Z::TSM && t < npts; t += Z::THREADS) {
            const int gg = t % G, qr = t / G, rr = qr % KY, q = qr / KY;
            const int a2 = a20 + rr;
            if (a2 >= g.H2) continue;
            const int kz = S * (q % D) + q / D;
            const int a3 = kz <= H ? kz : P3 - kz;
            const T s3 = kz <= H ? T(1) : T(-1);
            Ten6<T> tt;
            if (Z::TSM) {
                const T *tp = ten + (a3 * KY + rr) * G + gg;
                tt.xx = tp[0];
                tt.yy = tp[tstride];
                tt.zz = tp[2 * tstride];
                tt.xy = tp[3 * tstride];
                tt.xz = tp[4 * tstride] * s3;
                tt.yz = tp[5 * tstride] * s3;
            } else {
                const T *tp = b.Nk + ((long)a3 * g.H2 + a2) * g.Xp + kx0 + gg;
                const long tc = g.t_comp;
                tt.xx = __ldg(tp);
                tt.yy = __ldg(tp + tc);
                tt.zz = __ldg(tp + 2 * tc);
                tt.xy = __ldg(tp + 3 * tc);
                tt.xz = __ldg(tp + 4 * tc) * s3;
                tt.yz = __ldg(tp + 5 * tc) * s3;
            }
            Cx<T> *p = buf + q * nl + rr * G + gg;
            tensor_mul(tt, T(1), p, p + R2 * G, p + 2 * R2 * G);
            if (a2 > 0 && a2 < h2) {
                Cx<T> *pm = p + KY * G;
                tensor_mul(tt, T(-1), pm, pm + R2 * G, pm + 2 * R2 * G);
            }
        }
    }
    __syncthreads();
    {
        // inverse of part r, twisted by conj(w)^{mr}, back into the part's own (consumed) rows
        Cx<T> v[D];
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = buf[(r * D + k) * nl + l];
        f3::dft_reg<T, D, +1>(v);
#pragma unroll
        for (int m = 0; m < D; ++m) {
            Cx<T> u = v[f3::bitrev<D>(m)];
            if (r == 1) u = f3::rot<T, P3, +1>(u, m);
            else if (S == 4 && r == 2) u = f3::rot<T, P3, +1>(u, 2 * m);
            else if (S == 4 && r == 3) u = f3::rot<T, P3, +1>(u, 3 * m);
            buf[(r * D + m) * nl + l] = u;
        }
        __syncthreads();
        // z = r H/S + i, i < H/S (outputs z < H, shared by the S threads): z = m + jD
        const int gg = l % G, q = l / G, rw = q % R2, c = q / R2;
        const int ky = z_row_ky<KY>(g, a20, rw);
        if (ky >= 0) {
            Cx<T> *out = b.S + c * g.s_comp + (long)ky * g.Xp + kx0 + gg;
            const long zs = (long)g.P2 * g.Xp;
            constexpr int ZP = H / S;  // outputs per thread
#pragma unroll
            for (int i = 0; i < ZP; ++i) {
                const int z = r * ZP + i;
                if (z >= N3) break;
                const int m = z % D, j = z / D;  // j < S/2
                Cx<T> y = buf[m * nl + l];
#pragma unroll
                for (int rr = 1; rr < S; ++rr) {
                    const Cx<T> t = buf[(rr * D + m) * nl + l];
                    // conj(w_S)^{j rr}: (+i)^{j rr} for S = 4, (-1)^{j rr} for S = 2 (j = 0 there)
                    const int e = (j * rr) & (S - 1);
                    const Cx<T> tt = S == 2 ? t : (e == 0 ? t : (e == 1 ? mul_si(t, 1) : (e == 2 ? cx<T>(-t.x, -t.y) : mul_si(t, -1))));
                    y = f3::csum(y, tt);
                }
                out[z * zs] = y;
            }
        }
    }
}

// Single-layer variant (N3 == 1, P3 == 1): forward y, tensor product at kz = 0 (each octant row a2
// read once and applied to ky = a2 and P2 - a2), inverse y.  Lines l = c * G + g; element y of line l
// at buf[y * nl + l].  LG = 0 (N2 == 1): the product alone.
template <typename T, int LG>
__global__ void __launch_bounds__(kMaxThreadsYC<T>, 1) k_y_conv(Geom g, DemagBufs<T> b, int G)
{
    if (b.ctl && b.ctl->done) return;
    constexpr int P2 = 1 << LG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *buf = reinterpret_cast<Cx<T> *>(smem_raw);
    const int kx0 = blockIdx.x * G;
    const int nl = 3 * G;
    const int h2 = P2 >> 1;
    auto gaddr = [&](int c, int y) -> long { return c * g.s_comp + (long)y * g.Xp + kx0; };
    {
        const int rowb = G * (int)sizeof(Cx<T>);
        const int cb = rowb >= 16 ? 16 : rowb, lcpr = __ffs(rowb / cb) - 1;
        const int nrow = g.N2 * 3;
        for (int t = threadIdx.x; t < (nrow << lcpr); t += blockDim.x) {
            const int rr = t >> lcpr, ch = t - (rr << lcpr);
            const int y = rr / 3, c = rr - 3 * y;
            cpa_chunk((char *)(buf + y * nl + c * G) + ch * cb, (const char *)(b.S + gaddr(c, y)) + ch * cb, cb);
        }
        cpa_wait_all();
        __syncthreads();
    }
    const FastDiv nlf((unsigned)nl);
    if constexpr (LG > 0)
        f3::fft<T, LG, -1, true, true, true>(buf, nl, nlf, b.tw, g.twlg, g.N2, P2, f3::NoFn<T>(), f3::NoFn<T>());
    const int lG = __ffs(G) - 1;
    for (int t = threadIdx.x; t < G * g.H2; t += blockDim.x) {
        const int gg = t & (G - 1), a2 = t >> lG;
        const Ten6<T> ten = tensor_at(g, b, kx0 + gg, a2, 0);
        Cx<T> *p = buf + a2 * nl + gg;
        tensor_mul(ten, T(1), p, p + G, p + 2 * G);
        if (a2 > 0 && a2 < h2) {
            Cx<T> *pm = buf + (P2 - a2) * nl + gg;
            tensor_mul(ten, T(-1), pm, pm + G, pm + 2 * G);
        }
    }
    __syncthreads();
    auto dst = [&](int l, int y, Cx<T> v) {
        const int gg = l & (G - 1), c = l >> lG;
        b.S[gaddr(c, y) + gg] = v;
    };
    if constexpr (LG > 0) {
        f3::fft<T, LG, +1, true, true, false>(buf, nl, nlf, b.tw, g.twlg, P2, g.N2, f3::NoFn<T>(), dst);
    } else {
        for (int l = threadIdx.x; l < nl; l += blockDim.x) dst(l, 0, buf[l]);
    }
}

// ---------------------------------------------------------------------------------------------
static void set_smem(const void *f) { cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); }

template <typename T>
static void init_attributes_t()
{
    f3::lg_for_each<1, 10>([&](auto c) {
        constexpr int LG = decltype(c)::value;
        set_smem((const void *)k_x_fwd<T, false, LG>);
        set_smem((const void *)k_x_fwd<T, true, LG>);
        set_smem((const void *)k_x_inv<T, false, LG>);
        set_smem((const void *)k_x_inv<T, true, LG>);
    });
    f3::lg_for_each<1, 11>([&](auto c) {
        constexpr int LG = decltype(c)::value;
        set_smem((const void *)k_y_fwd<T, LG>);
        set_smem((const void *)k_y_inv<T, LG>);
    });
    f3::lg_for_each<1, 7>([&](auto c) {
        constexpr int LG = decltype(c)::value;
        set_smem((const void *)k_z_conv<T, LG>);
    });
    if constexpr (sizeof(T) == 4) {
        f3::lg_for_each<2, 6>([&](auto c) { set_smem((const void *)k_z_conv_r<decltype(c)::value>); });
    }
    f3::lg_for_each<0, 11>([&](auto c) {
        constexpr int LG = decltype(c)::value;
        set_smem((const void *)k_y_conv<T, LG>);
    });
}


static int pow2_floor(long v)
{
    if (v < 1) return 0;
    int p = 1;
    while (2L * p <= v) p *= 2;
    return p;
}
static int threads_for(long elems)
{
    long t = (elems + 7) / 8;
    t = t < 32 ? 32 : t;
    return (int)((t + 31) / 32 * 32);
}

// Launch shapes: every block transforms at most 8 complex values per thread; the y and z passes take
// up to kMaxThreads<T> threads so that their rows span at least 64 bytes where the size allows.
template <typename T>
DemagPlan demag_plan(const Geom &g)
{
    DemagPlan p{};
    p.ok = true;
    const size_t cs = sizeof(Cx<T>);
    const long budget = 8L * kMaxThreads<T>;
    if (g.P1 > 1) {
        const int xept = (sizeof(T) == 4 && g.lgQ >= 10) ? 16 : 8;
        int lpb = (int)((long)xept * kXThreads / g.Q);
        lpb = lpb > 64 ? 64 : lpb;
        if (lpb < 1 || g.lgQ > 10) p.ok = false;
        p.x_lpb = lpb < 1 ? 1 : lpb;
        p.x_threads = kXThreads;
        p.x_smem = (size_t)p.x_lpb * f3::padded(g.Q) * cs + (size_t)p.x_lpb * 3 * sizeof(int);
        int lpbi = (int)((long)xept * kXiThreads<T> / g.Q);  // the inverse takes the same stages (measured)
        lpbi = lpbi > 64 ? 64 : lpbi;
        if (lpbi < 1) p.ok = false;
        p.xi_lpb = lpbi < 1 ? 1 : lpbi;
        p.xi_threads = kXiThreads<T>;
        p.xi_smem = (size_t)p.xi_lpb * f3::padded(g.Q) * cs + (size_t)p.xi_lpb * 3 * sizeof(int);
    } else {
        p.x_lpb = 1;
        p.xi_lpb = 1;
        p.xi_threads = 256;
        p.xi_smem = 0;
        p.x_threads = 256;
        p.x_smem = 0;
    }
    if (g.N3 > 1) {
        // (P2 == 1: no y passes)
        p.y_G = 1;
        if (g.lgP2 > 11) p.ok = false;
        f3::lg_dispatch<1, 11>(g.lgP2, [&](auto c) {
            using Y = YTile<T, decltype(c)::value>;
            p.y_G = Y::G;
            p.y_threads = Y::THREADS;
            p.y_smem = Y::SMEM;
            p.yi_smem = Y::SMEM_TMA;
        });
        if (g.lgP3 < 1 || g.lgP3 > 7) p.ok = false;
        f3::lg_dispatch<1, 7>(g.lgP3, [&](auto c) {
            using Z = ZTile<T, decltype(c)::value>;
            p.z_G = Z::G;
            p.z_KY = Z::KY;
            p.z_threads = Z::THREADS;
            p.z_smem = Z::SMEM;
        });
        // FP32 lines of up to 64: the register z convolution
        p.z_reg = sizeof(T) == 4 && g.lgP3 >= 2 && g.lgP3 <= 6 && 2 * g.N3 <= g.P3;
        if (p.z_reg) {
            f3::lg_dispatch<2, 6>(g.lgP3, [&](auto c) {
                using Z = ZRTile<decltype(c)::value, kZRSplit<decltype(c)::value>>;
                p.z_G = Z::G;
                p.z_KY = Z::KY;
                p.z_threads = Z::THREADS;
                p.z_smem = Z::SMEM;
            });
        }
    } else {
        int G = pow2_floor(8L * kMaxThreadsYC<T> / (3L * g.P2));
        G = G > 16 ? 16 : G;
        if (G < 1 || g.lgP2 > 11) p.ok = false;
        p.yc_G = G < 1 ? 1 : G;
        p.yc_threads = threads_for(3L * p.yc_G * g.P2);
        p.yc_smem = (size_t)3 * p.yc_G * g.P2 * cs;
    }
    // every block holds at most (values per thread) x (threads) values of its transforms
    if (g.P1 > 1) {
        const long xept = (sizeof(T) == 4 && g.lgQ >= 10) ? 16 : 8;
        if ((long)p.x_lpb * g.Q > xept * p.x_threads || (long)p.xi_lpb * g.Q > xept * p.xi_threads) p.ok = false;
    }
    if (g.N3 > 1) {
        if (p.y_threads > kMaxThreads<T> * ((sizeof(T) == 4 && g.lgP2 >= 11) ? 2 : 1) ||
            p.z_threads > (p.z_reg ? 1024 : kMaxThreads<T>))
            p.ok = false;
    } else if (3L * p.yc_G * g.P2 > 8L * p.yc_threads || p.yc_threads > kMaxThreadsYC<T>) {
        p.ok = false;
    }
    // the kx grouping divides Xp (a multiple of 16)
    const int Gmax = g.N3 > 1 ? (p.y_G > p.z_G ? p.y_G : p.z_G) : p.yc_G;
    if (g.Xp % Gmax != 0) p.ok = false;
    if (p.x_smem > 200 * 1024 || p.xi_smem > 200 * 1024 || p.y_smem > 200 * 1024 || p.yi_smem > 200 * 1024 ||
        p.z_smem > 200 * 1024 || p.yc_smem > 200 * 1024)
        p.ok = false;
    return p;
}

// ---------------------------------------------------------------------------------------------
// TMA descriptor of a y-pass tile (the inverse pass's load, the forward pass's store) over
// S = [3][N3][P2][Xp] complex: every (component, z) plane holds P2 rows of Xp complex values (rows of
// Xp * sizeof(Cx<T>) bytes, a multiple of 128).  Dimensions in real elements, innermost first: the 2 Xp
// reals of a row, then (LFP = 3) the row within its group of 8 and the group, or (LFP = 0) the row, then
// the 3 N3 planes.  The box is the 2G reals of a block's G kx columns by all P2 rows of one plane: P2 / 8
// groups of 9 rows (the ninth outside the tensor, zero-filled by a load and skipped by a store: the
// padding row of the shared layout), or P2 plain rows.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled_fn()
{
    static EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return (EncodeTiledFn)f;
    }();
    return fn;
}

template <typename T>
int demag_encode_ymap(const Geom &g, void *S, CUtensorMap *map)
{
    memset(map, 0, sizeof(CUtensorMap));
    if (g.N3 <= 1 || g.P2 <= 1) return 0;  // no y passes
    const EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return -1;
    const DemagPlan p = demag_plan<T>(g);
    if (!p.ok) return -1;
    int LFP = 0;
    f3::lg_dispatch<1, 11>(g.lgP2, [&](auto c) { LFP = YTile<T, decltype(c)::value>::LFP; });
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const cuuint64_t rowb = (cuuint64_t)g.Xp * sizeof(Cx<T>);
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    CUresult r;
    if (LFP > 0) {
        const cuuint64_t dims[4] = {(cuuint64_t)2 * g.Xp, 8, (cuuint64_t)g.P2 / 8, (cuuint64_t)3 * g.N3};
        const cuuint64_t strides[3] = {rowb, 8 * rowb, (cuuint64_t)g.P2 * rowb};
        const cuuint32_t box[4] = {(cuuint32_t)(2 * p.y_G), 9, (cuuint32_t)(g.P2 / 8), 1};
        r = enc(map, dt, 4, S, dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[3] = {(cuuint64_t)2 * g.Xp, (cuuint64_t)g.P2, (cuuint64_t)3 * g.N3};
        const cuuint64_t strides[2] = {rowb, (cuuint64_t)g.P2 * rowb};
        const cuuint32_t box[3] = {(cuuint32_t)(2 * p.y_G), (cuuint32_t)g.P2, 1};
        r = enc(map, dt, 3, S, dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS ? 0 : (int)r;
}

template <typename T, bool CELL>
static void run_pipeline(const Geom &g, const DemagBufs<T> &b, const T *in, T *out, cudaStream_t st)
{
    const DemagPlan p = demag_plan<T>(g);
    if (!p.ok) return;
    // (create_mesh refuses shapes without a plan or, where there are y passes, without their descriptors)
    if (g.N3 > 1 && g.P2 > 1 && !b.ymap) return;
    const int nlines = 3 * g.N2 * g.N3;
    if (g.P1 == 1) {
        k_x_fwd1<T, CELL><<<div_up(nlines, 256), 256, 0, st>>>(g, b, in);
    } else {
        f3::lg_dispatch<1, 10>(g.lgQ, [&](auto c) {
            constexpr int LG = decltype(c)::value;
            k_x_fwd<T, CELL, LG><<<div_up(nlines, p.x_lpb), p.x_threads, p.x_smem, st>>>(g, b, in, p.x_lpb);
        });
    }
    b.mark("demag_x_fwd");
    if (g.N3 > 1) {
        if (g.P2 > 1) {
            f3::lg_dispatch<1, 11>(g.lgP2, [&](auto c) {
                constexpr int LG = decltype(c)::value;
                k_y_fwd<T, LG><<<dim3(g.Xp / p.y_G, 3 * g.N3), p.y_threads, p.yi_smem, st>>>(g, b, *b.ymap);
            });
            b.mark("demag_y_fwd");
        }
        if constexpr (sizeof(T) == 4) {
            if (p.z_reg) {
                f3::lg_dispatch<2, 6>(g.lgP3, [&](auto c) {
                    constexpr int LG = decltype(c)::value;
                    k_z_conv_r<LG><<<dim3(g.Xp / p.z_G, div_up(g.H2, p.z_KY)), p.z_threads, p.z_smem, st>>>(g, b);
                });
            }
        }
        if (!p.z_reg) {
            f3::lg_dispatch<1, 7>(g.lgP3, [&](auto c) {
                constexpr int LG = decltype(c)::value;
                k_z_conv<T, LG><<<dim3(g.Xp / p.z_G, div_up(g.H2, p.z_KY)), p.z_threads, p.z_smem, st>>>(g, b);
            });
        }
        b.mark("demag_z_conv");
        if (g.P2 > 1) {
            f3::lg_dispatch<1, 11>(g.lgP2, [&](auto c) {
                constexpr int LG = decltype(c)::value;
                k_y_inv<T, LG><<<dim3(g.Xp / p.y_G, 3 * g.N3), p.y_threads, p.yi_smem, st>>>(g, b, *b.ymap);
            });
            b.mark("demag_y_inv");
        }
    } else {
        f3::lg_dispatch<0, 11>(g.lgP2, [&](auto c) {
            constexpr int LG = decltype(c)::value;
            k_y_conv<T, LG><<<g.Xp / p.yc_G, p.yc_threads, p.yc_smem, st>>>(g, b, p.yc_G);
        });
        b.mark("demag_y_conv");
    }
    if (g.P1 == 1) {
        k_x_inv1<T, CELL><<<div_up(nlines, 256), 256, 0, st>>>(g, b, out);
    } else {
        f3::lg_dispatch<1, 10>(g.lgQ, [&](auto c) {
            constexpr int LG = decltype(c)::value;
            k_x_inv<T, CELL, LG><<<div_up(nlines, p.xi_lpb), p.xi_threads, p.xi_smem, st>>>(g, b, out, p.xi_lpb);
        });
    }
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

}  // namespace nm
