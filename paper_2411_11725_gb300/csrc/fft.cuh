// Block-level power-of-two FFT engine (Stockham autosort, radices 8, 4 and 2).
//
// Each thread keeps fft_regs<T>() complex values of the transform in registers per stage (one
// butterfly of the largest radix, or several smaller ones), so a length-2048 transform takes four stages.  The first stage reads its inputs through a caller functor (normally straight from global
// memory, skipping the zero padding) and the last stage writes through another functor (normally
// straight to global memory, skipping outputs nobody reads); only the exchanges between stages go
// through shared memory.  Shared-memory layouts insert one pad slot after every 16 elements so that
// the strided writes of the early stages do not collide in the same banks.
#pragma once
#include "nm_common.cuh"

namespace nm {

// twiddle table entry e^{-2 pi i k / 2^twlg}; inverse transforms use the conjugate
template <typename T>
__device__ __forceinline__ Cx<T> twiddle(const Cx<T> *__restrict__ tw, int idx, int dir)
{
    Cx<T> w = tw[idx];
    return dir < 0 ? w : conj(w);
}

// cos and sin of 2 pi k / 16 (k taken mod 16); constant-folded at every call site
__host__ __device__ constexpr double c16(int k)
{
    switch (k & 15) {
    case 0: return 1.0;
    case 1: case 15: return 0.92387953251128675613;
    case 2: case 14: return 0.70710678118654752440;
    case 3: case 13: return 0.38268343236508977173;
    case 4: case 12: return 0.0;
    case 5: case 11: return -0.38268343236508977173;
    case 6: case 10: return -0.70710678118654752440;
    case 7: case 9: return -0.92387953251128675613;
    default: return -1.0;
    }
}
__host__ __device__ constexpr double s16(int k) { return c16(k - 4); }

// x_k <- sum_j x_j e^{dir 2 pi i jk / R} in registers: in-place radix-2 decimation-in-frequency
// network; X_k ends up in x[bitrev(k)] (callers index with bitrev, a compile-time renaming).
template <int R>
__host__ __device__ constexpr int bitrev(int i)
{
    int r = 0;
    for (int b = 1, rb = R >> 1; b < R; b <<= 1, rb >>= 1)
        if (i & b) r |= rb;
    return r;
}

template <typename T, int R>
struct RegDft {
    __device__ __forceinline__ static void run(Cx<T> *x, int dir)
    {
#pragma unroll
        for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
            for (int s = 0; s < R; s += 2 * h) {
#pragma unroll
                for (int k = 0; k < h; ++k) {
                    const Cx<T> a = x[s + k], b = x[s + k + h];
                    x[s + k] = a + b;
                    const Cx<T> d = a - b;
                    const int q = k * (8 / h);  // W_{2h}^k = W_16^q
                    if (q == 0) x[s + k + h] = d;
                    else if (q == 4) x[s + k + h] = mul_si(d, dir);
                    else {
                        const T cq = (T)c16(q), sq = (T)s16(q);
                        x[s + k + h] = d * cx<T>(cq, dir > 0 ? sq : -sq);
                    }
                }
            }
        }
    }
};

// complex values per thread per stage (largest radix 8)
template <typename T>
__host__ __device__ constexpr int fft_regs()
{
    return 8;
}

// Asynchronous global -> shared copies (cp.async): many in flight per thread without registers.
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *sm, const void *gm)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(sm)), "l"(gm) : "memory");
}
__device__ __forceinline__ void cp_async8(void *sm, const void *gm)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(sm)), "l"(gm) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
// copy `bytes` (a multiple of 8, both addresses aligned to min(bytes, 16)) with cp.async
__device__ __forceinline__ void cp_async_row(void *sm, const void *gm, int bytes)
{
    char *d = (char *)sm;
    const char *s = (const char *)gm;
    if (bytes % 16 == 0)
        for (int o = 0; o < bytes; o += 16) cp_async16(d + o, s + o);
    else
        for (int o = 0; o < bytes; o += 8) cp_async8(d + o, s + o);
}

// Shared-memory slot of element i of a line with one pad slot per 16 elements.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int L) { return L + (L >> 4) + 1; }

// One Stockham stage of radix R on nl lines of length 2^lg, sub-transform length Ns = 2^slg.
//   src(l, i) -> value of input i of line l (only called for i < nin; larger i are zero)
//   dst(l, o, v) <- output o of line l (only called for o < nout)
//   SYNC_IN:  the source is shared memory also written by this stage: barrier between reads and writes
//   SYNC_OUT: barrier after the writes (the next stage reads them)
//   LF:       map consecutive threads to consecutive lines (layouts with lines innermost)
template <typename T, int R, bool LF, bool SYNC_IN, bool SYNC_OUT, typename Src, typename Dst>
__device__ __forceinline__ void fft_stage(const FastDiv &nlf, int lg, int slg, int dir, const Cx<T> *__restrict__ tw,
                                          int twlg, int nin, int nout, Src src, Dst dst)
{
    const int nl = (int)nlf.d;
    constexpr int lgR = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
    constexpr int BPT = fft_regs<T>() / R;
    const int L = 1 << lg, LR = L >> lgR;
    const int nb = nl * LR;
    const int Ns = 1 << slg;
    const int nt = blockDim.x;
    Cx<T> v[BPT][R];
#pragma unroll
    for (int c = 0; c < BPT; ++c) {
        const int b = threadIdx.x + c * nt;
        if (b < nb) {
            const int j = LF ? (int)nlf.div(b) : b & (LR - 1);
            const int l = LF ? b - j * nl : b >> (lg - lgR);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = j + r * LR;
                v[c][r] = i < nin ? src(l, i) : cx<T>(T(0), T(0));
            }
        }
    }
    if (SYNC_IN) __syncthreads();
#pragma unroll
    for (int c = 0; c < BPT; ++c) {
        const int b = threadIdx.x + c * nt;
        if (b < nb) {
            const int j = LF ? (int)nlf.div(b) : b & (LR - 1);
            const int l = LF ? b - j * nl : b >> (lg - lgR);
            const int k = j & (Ns - 1);
            if (k) {
                const int sh = twlg - slg - lgR;
#pragma unroll
                for (int r = 1; r < R; ++r) v[c][r] = v[c][r] * twiddle(tw, (k * r) << sh, dir);
            }
            RegDft<T, R>::run(v[c], dir);
            const int d = ((j >> slg) << (slg + lgR)) + k;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int o = d + r * Ns;
                if (o < nout) dst(l, o, v[c][bitrev<R>(r)]);
            }
        }
    }
    if (SYNC_OUT) __syncthreads();
}

// log2 radix of stage s (0-based) of a length-2^lg transform with largest radix 2^rmax: the remainder
// first, then the largest radix.
__host__ __device__ __forceinline__ int stage_lg(int lg, int s, int rmax)
{
    const int first = lg % rmax == 0 ? rmax : lg % rmax;
    return s == 0 ? first : rmax;
}
__host__ __device__ __forceinline__ int n_stages(int lg, int rmax) { return lg == 0 ? 0 : (lg + rmax - 1) / rmax; }

template <typename T, bool LF, bool SYNC_IN, bool SYNC_OUT, typename Src, typename Dst>
__device__ __forceinline__ void fft_stage_any(int rl, const FastDiv &nl, int lg, int slg, int dir,
                                              const Cx<T> *__restrict__ tw, int twlg, int nin, int nout, Src src,
                                              Dst dst)
{
    switch (rl) {
    case 4:
        if constexpr (fft_regs<T>() >= 16)
            fft_stage<T, 16, LF, SYNC_IN, SYNC_OUT>(nl, lg, slg, dir, tw, twlg, nin, nout, src, dst);
        break;
    case 3:
        if constexpr (fft_regs<T>() >= 8)
            fft_stage<T, 8, LF, SYNC_IN, SYNC_OUT>(nl, lg, slg, dir, tw, twlg, nin, nout, src, dst);
        break;
    case 2: fft_stage<T, 4, LF, SYNC_IN, SYNC_OUT>(nl, lg, slg, dir, tw, twlg, nin, nout, src, dst); break;
    default: fft_stage<T, 2, LF, SYNC_IN, SYNC_OUT>(nl, lg, slg, dir, tw, twlg, nin, nout, src, dst); break;
    }
}

// Whole transform: first stage from `src` (inputs >= nin are zero), middle stages in place in the
// shared buffer addressed by `sm(l, i)`, last stage to `dst` (outputs >= nout dropped).
// SRC_SM / DST_SM: src / dst are the same shared buffer (barriers are then placed around them); the
// caller synchronises before a shared-memory source.  Needs nl * 2^lg <= fft_regs<T>() * blockDim.x.
template <typename T, bool LF, bool SRC_SM, bool DST_SM, typename Src, typename SmAddr, typename Dst>
__device__ __forceinline__ void fft_lines(Cx<T> *buf, const FastDiv &nlf, int lg, int dir, const Cx<T> *__restrict__ tw,
                                          int twlg, int nin, int nout, Src src, SmAddr sm, Dst dst)
{
    const int nl = (int)nlf.d;
    auto sm_src = [&](int l, int i) { return buf[sm(l, i)]; };
    auto sm_dst = [&](int l, int i, Cx<T> v) { buf[sm(l, i)] = v; };
    constexpr int rmax = fft_regs<T>() == 16 ? 4 : (fft_regs<T>() == 8 ? 3 : 2);
    const int ns = n_stages(lg, rmax);
    if (ns == 0) {
        // length 1: copy through registers
        Cx<T> v[fft_regs<T>()];
#pragma unroll
        for (int c = 0; c < fft_regs<T>(); ++c) {
            int l = threadIdx.x + c * blockDim.x;
            if (l < nl) v[c] = nin > 0 ? src(l, 0) : cx<T>(T(0), T(0));
        }
        if (SRC_SM && DST_SM) __syncthreads();
#pragma unroll
        for (int c = 0; c < fft_regs<T>(); ++c) {
            int l = threadIdx.x + c * blockDim.x;
            if (l < nl && nout > 0) dst(l, 0, v[c]);
        }
        if (DST_SM) __syncthreads();
        return;
    }
    if (ns == 1) {
        fft_stage_any<T, LF, SRC_SM && DST_SM, DST_SM>(stage_lg(lg, 0, rmax), nlf, lg, 0, dir, tw, twlg, nin, nout, src,
                                                        dst);
        return;
    }
    int slg = 0;
    for (int s = 0; s < ns; ++s) {
        const int rl = stage_lg(lg, s, rmax);
        if (s == 0)
            fft_stage_any<T, LF, SRC_SM, true>(rl, nlf, lg, slg, dir, tw, twlg, nin, 1 << lg, src, sm_dst);
        else if (s + 1 < ns)
            fft_stage_any<T, LF, true, true>(rl, nlf, lg, slg, dir, tw, twlg, 1 << lg, 1 << lg, sm_src, sm_dst);
        else
            fft_stage_any<T, LF, DST_SM, DST_SM>(rl, nlf, lg, slg, dir, tw, twlg, 1 << lg, nout, sm_src, dst);
        slg += rl;
    }
}

}  // namespace nm
