// Block-level power-of-two FFT on lines held in shared memory (Stockham autosort, radix 4 with one
// radix-2 stage when log2 L is odd).  Used by every demag pass: the lines of a pass are staged in
// shared memory by the pass (with its own fused pre- and post-processing) and transformed in place.
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

// In-place unnormalised DFT of `nl` lines of length L = 2^lg at buf[l*ls + i], i < L.
// dir = -1: X_k = sum_j x_j e^{-2 pi i jk/L}; dir = +1: the same with e^{+...}.
// Every thread of the block must call it; MAXB bounds the radix-4 butterflies per thread per stage:
// the caller guarantees nl * L / 4 <= MAXB * blockDim.x.
template <typename T, int MAXB>
__device__ void smem_fft(Cx<T> *buf, int nl, int ls, int lg, int dir, const Cx<T> *__restrict__ tw, int twlg)
{
    if (lg == 0) return;
    const int L = 1 << lg;
    const int nt = blockDim.x, tid = threadIdx.x;
    int slg = 0;  // log2 of the current sub-transform length Ns
    if (lg & 1) {
        // radix-2 first stage (Ns = 1: no twiddles)
        const int half = L >> 1, nb = nl * half;
        Cx<T> v0[2 * MAXB], v1[2 * MAXB];
#pragma unroll
        for (int c = 0; c < 2 * MAXB; ++c) {
            int b = tid + c * nt;
            if (b < nb) {
                int l = b >> (lg - 1), j = b & (half - 1);
                v0[c] = buf[l * ls + j];
                v1[c] = buf[l * ls + j + half];
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 2 * MAXB; ++c) {
            int b = tid + c * nt;
            if (b < nb) {
                int l = b >> (lg - 1), j = b & (half - 1);
                buf[l * ls + 2 * j] = v0[c] + v1[c];
                buf[l * ls + 2 * j + 1] = v0[c] - v1[c];
            }
        }
        __syncthreads();
        slg = 1;
    }
    const int quarter = L >> 2;
    for (; slg < lg; slg += 2) {
        const int nb = nl * quarter;
        const int Ns = 1 << slg;
        const int tsh = twlg - slg - 2;  // twiddle index = k*r << tsh
        Cx<T> v[MAXB][4];
#pragma unroll
        for (int c = 0; c < MAXB; ++c) {
            int b = tid + c * nt;
            if (b < nb) {
                int l = b >> (lg - 2), j = b & (quarter - 1);
                const Cx<T> *src = buf + l * ls + j;
                v[c][0] = src[0];
                v[c][1] = src[quarter];
                v[c][2] = src[2 * quarter];
                v[c][3] = src[3 * quarter];
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < MAXB; ++c) {
            int b = tid + c * nt;
            if (b < nb) {
                int l = b >> (lg - 2), j = b & (quarter - 1);
                int k = j & (Ns - 1);
                Cx<T> a0 = v[c][0], a1 = v[c][1], a2 = v[c][2], a3 = v[c][3];
                if (k) {
                    a1 = a1 * twiddle(tw, k << tsh, dir);
                    a2 = a2 * twiddle(tw, (2 * k) << tsh, dir);
                    a3 = a3 * twiddle(tw, (3 * k) << tsh, dir);
                }
                Cx<T> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = mul_si(a1 - a3, dir);
                int d = ((j >> slg) << (slg + 2)) + k;
                Cx<T> *dst = buf + l * ls + d;
                dst[0] = t0 + t2;
                dst[Ns] = t1 + t3;
                dst[2 * Ns] = t0 - t2;
                dst[3 * Ns] = t1 - t3;
            }
        }
        __syncthreads();
    }
}

}  // namespace nm
