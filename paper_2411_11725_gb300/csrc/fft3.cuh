// Block-level power-of-two FFT engine with the transform length fixed at compile time.
//
// A length-2^LG transform runs as Stockham stages: a first stage of the remainder radix, then radix-8
// (or radix-16) stages.  Each thread keeps 8 (or 16) complex values in registers per stage (one
// butterfly of the largest radix, or several smaller ones).  Because LG, the radices, the sub-transform
// lengths and the direction are template constants, every index of a stage reduces to shifts, masks
// and immediate offsets.  The first stage reads its inputs through a caller functor or from shared
// memory, and the last stage writes through a functor or to shared memory; only the exchanges between
// stages go through shared memory.
//
// Shared-memory layouts of a block's nl lines:
//   LF (lines fastest):  element i of line l at buf[lfpad(i) * nl + l], lfpad(i) = i + (i >> LFP) with
//                        one padding row every 2^LFP elements when LFP > 0 (consecutive threads take
//                        consecutive lines; the padding rows break the strided bank pattern of the first
//                        stage's stores when a block holds only a few lines)
//   line-major:          element i of line l at buf[l * LSZ + pad16(i)], LSZ = padded_len(2^LG)
//                        (one pad slot per 16 elements breaks the strided bank pattern of the early
//                        stages)
#pragma once
#include <type_traits>

#include "nm_common.cuh"

namespace nm {
namespace f3 {

// Stage plan of a length-2^LG transform with at most 2^RM values per butterfly (RM = 3: radix 8,
// RM = 4: radix 16): the remainder radix first, then radix 2^RM.
__host__ __device__ constexpr int first_lg(int LG, int RM = 3) { return LG % RM == 0 ? RM : LG % RM; }
__host__ __device__ constexpr int n_stages(int LG, int RM = 3) { return LG == 0 ? 0 : 1 + (LG - first_lg(LG, RM)) / RM; }
__host__ __device__ constexpr int stage_lg(int LG, int s, int RM = 3) { return s == 0 ? first_lg(LG, RM) : RM; }
__host__ __device__ constexpr int stage_slg(int LG, int s, int RM = 3)
{
    return s == 0 ? 0 : first_lg(LG, RM) + RM * (s - 1);
}

__host__ __device__ constexpr int pad16c(int i) { return i + (i >> 4); }
template <int LFP>
__host__ __device__ constexpr int lfpad(int i) { return LFP > 0 ? i + (i >> LFP) : i; }
// rows of the LF layout for lines of L elements
__host__ __device__ constexpr int lf_rows(int L, int LFP) { return LFP > 0 ? L + (L >> LFP) : L; }
__host__ __device__ constexpr int padded(int L) { return L + (L >> 4) + 1; }

// cos and sin of 2 pi k / 16 (k mod 16), folded to constants at each call site
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
// the same cosines as a table of the working precision (indexed with unrolled constants)
template <typename T>
__device__ constexpr T kC16[16] = {(T)c16(0),  (T)c16(1),  (T)c16(2),  (T)c16(3), (T)c16(4),  (T)c16(5),
                                   (T)c16(6),  (T)c16(7),  (T)c16(8),  (T)c16(9), (T)c16(10), (T)c16(11),
                                   (T)c16(12), (T)c16(13), (T)c16(14), (T)c16(15)};

template <int R>
__host__ __device__ constexpr int bitrev(int i)
{
    int r = 0;
    for (int b = 1, rb = R >> 1; b < R; b <<= 1, rb >>= 1)
        if (i & b) r |= rb;
    return r;
}

// FP32 complex sum and difference as packed pairs (add.rn.f32x2 / sub.rn.f32x2: one instruction for
// both parts, rounded exactly as the scalar additions)
__device__ __forceinline__ unsigned long long pack2(Cx<float> a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ Cx<float> unpack2(unsigned long long r)
{
    Cx<float> a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
template <typename T>
__device__ __forceinline__ Cx<T> csum(Cx<T> a, Cx<T> b)
{
    if constexpr (sizeof(T) == 4) {
        unsigned long long d;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(a)), "l"(pack2(b)));
        return unpack2(d);
    } else {
        return a + b;
    }
}
template <typename T>
__device__ __forceinline__ Cx<T> cdiff(Cx<T> a, Cx<T> b)
{
    if constexpr (sizeof(T) == 4) {
        unsigned long long d;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(a)), "l"(pack2(b)));
        return unpack2(d);
    } else {
        return a - b;
    }
}

// x_k <- sum_j x_j e^{DIR 2 pi i jk / R}: radix-2 decimation-in-frequency network, X_k in x[bitrev(k)]
template <typename T, int R, int DIR, bool PK = true>
__device__ __forceinline__ void dft(Cx<T> *x)
{
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int s = 0; s < R; s += 2 * h) {
#pragma unroll
            for (int k = 0; k < h; ++k) {
                const Cx<T> a = x[s + k], b = x[s + k + h];
                x[s + k] = PK ? csum(a, b) : a + b;
                const Cx<T> d = PK ? cdiff(a, b) : a - b;
                const int q = k * (8 / h);  // W_{2h}^k = W_16^q
                if (q == 0) x[s + k + h] = d;
                else if (q == 4) x[s + k + h] = mul_si(d, DIR);
                else {
                    const T cq = kC16<T>[q & 15], sq = DIR > 0 ? kC16<T>[(q - 4) & 15] : -kC16<T>[(q - 4) & 15];
                    x[s + k + h] = cx<T>(d.x * cq - d.y * sq, d.x * sq + d.y * cq);
                }
            }
        }
    }
}

// cos(2 pi num / den) at compile time: reflection to an angle in [0, pi/4] and a Taylor series there
// (14 terms: far below double rounding), for the constants of the in-register transforms below
__host__ __device__ constexpr double taylor_cos(double x)
{
    double t = 1.0, s = 1.0;
    for (int k = 1; k < 14; ++k) {
        t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        s += t;
    }
    return s;
}
__host__ __device__ constexpr double taylor_sin(double x)
{
    double t = x, s = x;
    for (int k = 1; k < 14; ++k) {
        t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        s += t;
    }
    return s;
}
__host__ __device__ constexpr double cos2pi(int num, int den)
{
    constexpr double kPi = 3.14159265358979323846;
    num = ((num % den) + den) % den;
    if (2 * num > den) num = den - num;  // cos(2 pi f) = cos(2 pi (1 - f)): angle in [0, pi]
    const double x = 2.0 * kPi * (double)num / (double)den;
    if (x > 0.5 * kPi) {
        const double y = kPi - x;  // cos x = -cos(pi - x)
        return y > 0.25 * kPi ? -taylor_sin(0.5 * kPi - y) : -taylor_cos(y);
    }
    return x > 0.25 * kPi ? taylor_sin(0.5 * kPi - x) : taylor_cos(x);
}
template <typename T, int N>
struct CosTab {
    T v[N];
};
template <typename T, int N>
__host__ __device__ constexpr CosTab<T, N> make_cos_tab()
{
    CosTab<T, N> t{};
    for (int k = 0; k < N; ++k) t.v[k] = (T)cos2pi(k, N);
    return t;
}
// cos(2 pi k / N), k < N, in the working precision (indexed with unrolled constants)
template <typename T, int N>
__device__ constexpr CosTab<T, N> kCos = make_cos_tab<T, N>();

// v * e^{DIR 2 pi i k / N} with k a compile-time constant after unrolling
template <typename T, int N, int DIR>
__device__ __forceinline__ Cx<T> rot(Cx<T> v, int k)
{
    k &= N - 1;
    if (k == 0) return v;
    if (4 * k == N) return mul_si(v, DIR);
    if (4 * k == 3 * N) return mul_si(v, -DIR);
    if (2 * k == N) return cx<T>(-v.x, -v.y);
    const T c = kCos<T, N>.v[k], s = DIR > 0 ? kCos<T, N>.v[(k - N / 4) & (N - 1)] : -kCos<T, N>.v[(k - N / 4) & (N - 1)];
    return cx<T>(v.x * c - v.y * s, v.x * s + v.y * c);
}

// A whole transform of R <= 32 values held by one thread: X_k = sum_j x_j e^{DIR 2 pi i jk / R}, X_k in
// x[bitrev(k)].  R = 32 splits into one radix-2 decimation-in-frequency level and two 16-point networks.
template <typename T, int R, int DIR>
__device__ __forceinline__ void dft_reg(Cx<T> *x);

// v * conj^(DIR>0)(w): the twiddle table holds e^{-2 pi i k / 2^twlg}
template <typename T, int DIR>
__device__ __forceinline__ Cx<T> twmul(Cx<T> v, Cx<T> w)
{
    if (DIR < 0) return cx<T>(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
    return cx<T>(v.x * w.x + v.y * w.y, v.y * w.x - v.x * w.y);
}

// packed additions in the in-register transforms too (measured faster than scalar ones)
constexpr bool kRegPacked = true;
template <typename T, int R, int DIR>
__device__ __forceinline__ void dft_reg(Cx<T> *x)
{
    static_assert(R >= 1 && R <= 32 && (R & (R - 1)) == 0, "in-register transforms of 1 to 32 values");
    if constexpr (R == 32) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const Cx<T> a = x[k], b = x[k + 16];
            x[k] = kRegPacked ? csum(a, b) : a + b;
            x[k + 16] = rot<T, 32, DIR>(kRegPacked ? cdiff(a, b) : a - b, k);
        }
        dft<T, 16, DIR, kRegPacked>(x);
        dft<T, 16, DIR, kRegPacked>(x + 16);
    } else if constexpr (R > 1) {
        dft<T, R, DIR, kRegPacked>(x);
    }
}

// Input / output modes of a stage
enum { IN_FN = 0, IN_SM = 1 };
enum { OUT_FN = 0, OUT_SM = 1 };

// One stage S of a length-2^LG transform on nl lines (nb = nl * 2^LG / R butterflies).
template <typename T, int LG, int S, int DIR, bool LF, int IN, int OUT, bool SYNC_IN, bool SYNC_OUT, int EPT,
          int NLC, int LFP, typename Src, typename Dst>
__device__ __forceinline__ void stage(Cx<T> *__restrict__ buf, int nl_rt, const FastDiv &nlf,
                                      const Cx<T> *__restrict__ tw, int twlg, int nin, int nout, const Src &src,
                                      const Dst &dst)
{
    const int nl = NLC > 0 ? NLC : nl_rt;  // a compile-time line count turns the index arithmetic into constants
    constexpr int RM = EPT == 16 ? 4 : 3;
    constexpr int RLG = stage_lg(LG, S, RM), R = 1 << RLG, SLG = stage_slg(LG, S, RM), NS = 1 << SLG;
    constexpr int L = 1 << LG, LR = L >> RLG, LSZ = padded(L), BPT = EPT / R;
    const int nb = nl * LR;
    Cx<T> v[BPT][R];
    int jv[BPT], lv[BPT];
#pragma unroll
    for (int c = 0; c < BPT; ++c) {
        const int b = threadIdx.x + c * blockDim.x;
        int j, l;
        if (LF) {
            j = NLC > 0 ? b / NLC : (int)nlf.div((unsigned)b);
            l = b - j * nl;
        } else {
            j = b & (LR - 1);
            l = b >> (LG - RLG);
        }
        jv[c] = j;
        lv[c] = l;
        if (b < nb) {
            if (IN == IN_FN) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = j + r * LR;
                    v[c][r] = (S > 0 || i < nin) ? src(l, i) : cx<T>(T(0), T(0));
                }
            } else if (LF) {
                // element j + r LR: lfpad folds into a constant step when LR is a multiple of 2^LFP
                constexpr bool fold = LFP == 0 || LR % (1 << (LFP > 0 ? LFP : 0)) == 0;
                const Cx<T> *p = buf + lfpad<LFP>(j) * nl + l;
                const int step = lf_rows(LR, LFP) * nl;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = j + r * LR;
                    v[c][r] = (S > 0 || i < nin) ? (fold ? p[r * step] : buf[lfpad<LFP>(i) * nl + l])
                                                 : cx<T>(T(0), T(0));
                }
            } else {
                const Cx<T> *p = buf + l * LSZ;
                const int pj = pad16c(j);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = j + r * LR;
                    const int a = (LR % 16 == 0) ? pj + r * (LR + LR / 16) : pad16c(i);
                    v[c][r] = (S > 0 || i < nin) ? p[a] : cx<T>(T(0), T(0));
                }
            }
        }
    }
    if (SYNC_IN) __syncthreads();
    const int sh = twlg - SLG - RLG;
#pragma unroll
    for (int c = 0; c < BPT; ++c) {
        const int b = threadIdx.x + c * blockDim.x;
        if (b >= nb) continue;
        const int j = jv[c], l = lv[c];
        const int k = j & (NS - 1);
        if (NS > 1) {
            const int kk = k << sh;
            if constexpr (R == 16 && sizeof(T) == 4) {
                // w^r for r < 16 from the four table values w, w^2, w^4, w^8 (four loads in flight together
                // instead of fifteen; the other powers are at most three products away, a few roundings).
                // FP32 only: the FP64 passes are bound by the FP64 rate, where the products cost more than
                // the loads they save.
                Cx<T> w[16];
                w[1] = tw[kk];
                w[2] = tw[2 * kk];
                w[4] = tw[4 * kk];
                w[8] = tw[8 * kk];
                w[3] = w[1] * w[2];
                w[5] = w[4] * w[1];
                w[6] = w[4] * w[2];
                w[7] = w[4] * w[3];
#pragma unroll
                for (int r = 9; r < 16; ++r) w[r] = w[8] * w[r - 8];
#pragma unroll
                for (int r = 1; r < R; ++r) v[c][r] = twmul<T, DIR>(v[c][r], w[r]);
            } else {
#pragma unroll
                for (int r = 1; r < R; ++r) v[c][r] = twmul<T, DIR>(v[c][r], tw[kk * r]);
            }
        }
        dft<T, R, DIR>(v[c]);
        const int d = ((j >> SLG) << (SLG + RLG)) + k;
        if (OUT == OUT_FN) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int o = d + r * NS;
                if (o < nout) dst(l, o, v[c][bitrev<R>(r)]);
            }
        } else if (LF) {
            constexpr bool fold = LFP == 0 || NS % (1 << (LFP > 0 ? LFP : 0)) == 0;
            Cx<T> *p = buf + lfpad<LFP>(d) * nl + l;
            const int step = lf_rows(NS, LFP) * nl;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (fold) p[r * step] = v[c][bitrev<R>(r)];
                else buf[lfpad<LFP>(d + r * NS) * nl + l] = v[c][bitrev<R>(r)];
            }
        } else {
            Cx<T> *p = buf + l * LSZ;
            const int pd = pad16c(d);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int a = (NS % 16 == 0) ? pd + r * (NS + NS / 16) : pad16c(d + r * NS);
                p[a] = v[c][bitrev<R>(r)];
            }
        }
    }
    if (SYNC_OUT) __syncthreads();
}

template <typename T, int LG, int S, int DIR, bool LF, bool SRC_SM, bool DST_SM, int EPT, int NLC, int LFP,
          typename Src, typename Dst>
__device__ __forceinline__ void run_stages(Cx<T> *buf, int nl, const FastDiv &nlf, const Cx<T> *__restrict__ tw,
                                           int twlg, int nin, int nout, const Src &src, const Dst &dst)
{
    constexpr int NSG = n_stages(LG, EPT == 16 ? 4 : 3);
    if constexpr (S < NSG) {
        constexpr bool first = S == 0, last = S + 1 == NSG;
        constexpr int IN = (first && !SRC_SM) ? IN_FN : IN_SM;
        constexpr int OUT = (last && !DST_SM) ? OUT_FN : OUT_SM;
        constexpr bool SYNC_IN = IN == IN_SM && OUT == OUT_SM;  // in place: all reads before any write
        constexpr bool SYNC_OUT = OUT == OUT_SM;
        stage<T, LG, S, DIR, LF, IN, OUT, SYNC_IN, SYNC_OUT, EPT, NLC, LFP>(
            buf, nl, nlf, tw, twlg, first ? nin : (1 << LG), last ? nout : (1 << LG), src, dst);
        run_stages<T, LG, S + 1, DIR, LF, SRC_SM, DST_SM, EPT, NLC, LFP>(buf, nl, nlf, tw, twlg, nin, nout, src, dst);
    }
}

// Transform nl lines of length 2^LG (LG >= 1): inputs i >= nin are zero, outputs o >= nout dropped.
// SRC_SM: the first stage reads the shared layout (the caller synchronised after filling it);
// otherwise src(l, i) is called for i < nin.  DST_SM: the last stage writes the shared layout
// (followed by a barrier); otherwise dst(l, o, v) is called for o < nout.
// EPT (8 or 16) values per thread per stage: needs nl * 2^LG <= EPT * blockDim.x.  NLC > 0: the line
// count is the compile-time constant NLC (nl and nlf are then ignored).  LFP: row padding of the LF layout.
template <typename T, int LG, int DIR, bool LF, bool SRC_SM, bool DST_SM, int EPT = 8, int NLC = 0, int LFP = 0,
          typename Src, typename Dst>
__device__ __forceinline__ void fft(Cx<T> *buf, int nl, const FastDiv &nlf, const Cx<T> *__restrict__ tw, int twlg,
                                    int nin, int nout, const Src &src, const Dst &dst)
{
    static_assert(LG >= 1, "length-1 transforms are copies");
    static_assert(EPT == 8 || EPT == 16, "8 or 16 values per thread");
    static_assert(LF || LFP == 0, "row padding belongs to the lines-fastest layout");
    run_stages<T, LG, 0, DIR, LF, SRC_SM, DST_SM, EPT, NLC, LFP>(buf, nl, nlf, tw, twlg, nin, nout, src, dst);
}

// placeholder functor for a stage side that is shared memory
template <typename T>
struct NoFn {
    __device__ Cx<T> operator()(int, int) const { return cx<T>(T(0), T(0)); }
    __device__ void operator()(int, int, Cx<T>) const {}
};

// Compile-time dispatch of a runtime log2 length in [LO, HI]
template <int LO, int HI, typename F>
inline bool lg_dispatch(int lg, F &&f)
{
    if constexpr (LO <= HI) {
        if (lg == LO) {
            f(std::integral_constant<int, LO>{});
            return true;
        }
        return lg_dispatch<LO + 1, HI>(lg, f);
    } else {
        return false;
    }
}
template <int LO, int HI, typename F>
inline void lg_for_each(F &&f)
{
    if constexpr (LO <= HI) {
        f(std::integral_constant<int, LO>{});
        lg_for_each<LO + 1, HI>(f);
    }
}

}  // namespace f3
}  // namespace nm
