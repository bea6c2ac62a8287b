// Runge-Kutta bookkeeping kernels: stage inputs, Dormand-Prince error norm with a deterministic
// two-level reduction, device-side step control, the accepted update with renormalisation, and the
// boundary layout conversions.
#include "rk.cuh"

namespace nm {

constexpr int kRedThreads = 256;

// y = m + dt * sum_j a_j k_j: slope combination in the working precision, addition in FP64
// (with mf, the FP32 path forms y = fl32(m) + dt * sum in FP32: y is an FP32 quantity either way)
template <typename T>
__global__ void k_stage_input(long n_nodes, long ns, const double *__restrict__ m, KList k, const StepCtl *ctl,
                              T *__restrict__ y, const float *__restrict__ mf)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    if (ctl->done) return;
    const double dt = ctl->dt;
    for (int c = 0; c < 3; ++c) {
        long i = c * ns + n;
        T acc = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j >= k.n) break;
            acc += kcoef<T>(k, j) * ((const T *)k.p[j])[i];
        }
        if (sizeof(T) == 4 && mf) y[i] = (T)(mf[i] + (float)dt * (float)acc);
        else y[i] = (T)(m[i] + dt * (double)acc);
    }
}

// The FP32 stage input with the FP32 copy of m, four consecutive nodes per thread (16-byte vectors);
// thread q also forms node 4 n4 + q of the ragged tail (q < n_nodes mod 4)
__global__ void k_stage_input_f4(long n_nodes, long ns, KList k, const StepCtl *ctl, float *__restrict__ y,
                                 const float *__restrict__ mf)
{
    const long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (ctl->done) return;
    const float dtf = (float)ctl->dt;
    const long n4 = n_nodes >> 2;
    if (q < n4) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j >= k.n) break;
                const float4 v = reinterpret_cast<const float4 *>((const float *)k.p[j] + c * ns)[q];
                const float a = k.af[j];
                acc.x += a * v.x; acc.y += a * v.y; acc.z += a * v.z; acc.w += a * v.w;
            }
            const float4 m = reinterpret_cast<const float4 *>(mf + c * ns)[q];
            reinterpret_cast<float4 *>(y + c * ns)[q] =
                make_float4(m.x + dtf * acc.x, m.y + dtf * acc.y, m.z + dtf * acc.z, m.w + dtf * acc.w);
        }
    }
    if (q < (n_nodes & 3)) {
        const long n = 4 * n4 + q;
        for (int c = 0; c < 3; ++c) {
            const long i = c * ns + n;
            float acc = 0.f;
            for (int j = 0; j < 8; ++j) {
                if (j >= k.n) break;
                acc += k.af[j] * ((const float *)k.p[j])[i];
            }
            y[i] = mf[i] + dtf * acc;
        }
    }
}

// 1/sqrt(s) for s > 0 in FP64 from an FP32 estimate and one Newton step (relative error ~1e-14), so
// the FP32 path renormalises without FP64 division or square root.
__device__ __forceinline__ double rsqrt_refined(double s)
{
    const double r0 = (double)rsqrtf((float)s);
    return r0 * (1.5 - 0.5 * s * r0 * r0);
}

template <typename T>
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// Per-block partial sums of ((dt sum_i e_i k_i) / (atol + rtol max(|m|, |m5|)))^2 over magnetic
// nodes, m5 = m + dt sum_i b_i k_i.  The per-node terms follow the working precision of the slopes
// (F64T: in FP64 for FP32 slopes too, from the FP64 m and FP64 coefficients); the sums are FP64.
template <typename T, bool F64T = false>
__global__ void __launch_bounds__(kRedThreads) k_dp5_err(long n_nodes, long ns, const double *__restrict__ m,
                                                          KList kb, KList ke, const T *__restrict__ inv_mass,
                                                          const StepCtl *ctl, double *partials,
                                                          const float *__restrict__ mf)
{
    __shared__ double sh[kRedThreads];
    if (ctl->done) return;
    const double dt = ctl->dt, rtol = ctl->rtol, atol = ctl->atol;
    double acc = 0.0;
    // no early exit per node: all loads of an iteration are independent, so they are in flight together
#pragma unroll 2
    for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < n_nodes; n += (long)gridDim.x * blockDim.x) {
        const bool magnetic = inv_mass[n] > T(0);
        T part = 0;
        for (int c = 0; c < 3; ++c) {
            long i = c * ns + n;
            if (F64T && sizeof(T) == 4) {
                // every operation of the term in FP64 (the FP32 slopes are exact in FP64)
                double db = 0.0, de = 0.0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (j >= kb.n) break;
                    const double kv = (double)((const T *)kb.p[j])[i];
                    db += kb.a[j] * kv;
                    de += ke.a[j] * kv;
                }
                const double m0 = m[i], m5 = m0 + dt * db;
                const double sc = atol + rtol * fmax(fabs(m0), fabs(m5));
                const double q = dt * de / sc;
                acc += magnetic ? q * q : 0.0;
                continue;
            }
            T sb = 0, se = 0, k1v = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j >= kb.n) break;
                const T kv = ((const T *)kb.p[j])[i];
                sb += kcoef<T>(kb, j) * kv;
                if (sizeof(T) == 8) {
                    se += kcoef<T>(ke, j) * kv;
                } else if (j == 0) {
                    k1v = kv;
                } else {
                    se += kcoef<T>(ke, j) * (kv - k1v);  // difference form (see dp5_err_term)
                }
            }
            if (sizeof(T) == 8) {
                const double m0 = m[i], m5 = m0 + dt * (double)sb;
                const double sc = atol + rtol * fmax(fabs(m0), fabs(m5));
                const double q = dt * (double)se / sc;
                acc += magnetic ? q * q : 0.0;
            } else {
                // the error scale only weights the norm: FP32 is ample for max(|m|, |m5|)
                const float m0 = mf ? mf[i] : (float)m[i], dtf = (float)dt;
                const float m5 = m0 + dtf * (float)sb;
                const float sc = (float)atol + (float)rtol * fmaxf(fabsf(m0), fabsf(m5));
                const float q = __fdividef(dtf * (float)se, sc);  // a weight of the norm: fast division
                part += (T)(q * q);
            }
        }
        if (sizeof(T) == 4 && magnetic) acc += (double)part;
    }
    double s = block_sum<T>(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// FP32 slopes with the FP32 copy of m: the same partial sums with four consecutive nodes per thread and
// load (16-byte vectors; every component array starts on a 256-byte boundary), fewer and longer
// requests for the 25 streams the norm reads.  Nodes past the last full group of four go through the
// scalar terms of block 0.
//
// The error combination sum_j e_j k_j (e_j = b_j - b*_j, first slope k_1) is formed in FP32 as
// sum_{j>1} e_j (k_j - k_1).  The weights sum to zero, so this is the same quantity; the slopes of one
// step are close to each other, so their differences are exact in FP32 and the combination keeps its
// relative accuracy when it is far smaller than the slopes (small steps), where the direct sum with
// FP32-rounded weights would leave a residue of about 1e-8 |k_1|.
__device__ __forceinline__ float dp5_err_term(float m0, float sb, float se, float dtf, float rtol, float atol)
{
    const float m5 = m0 + dtf * sb;
    const float sc = atol + rtol * fmaxf(fabsf(m0), fabsf(m5));
    const float q = __fdividef(dtf * se, sc);  // a weight of the norm: fast division
    return q * q;
}

__global__ void __launch_bounds__(kRedThreads) k_dp5_err_f4(long n_nodes, long ns, KList kb, KList ke,
                                                             const float *__restrict__ inv_mass, const StepCtl *ctl,
                                                             double *partials, const float *__restrict__ mf)
{
    __shared__ double sh[kRedThreads];
    if (ctl->done) return;
    const float dtf = (float)ctl->dt, rtol = (float)ctl->rtol, atol = (float)ctl->atol;
    double acc = 0.0;
    const long n4 = n_nodes >> 2;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n4; q += (long)gridDim.x * blockDim.x) {
        const float4 im = reinterpret_cast<const float4 *>(inv_mass)[q];
        float4 part = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 sb = make_float4(0.f, 0.f, 0.f, 0.f), se = sb, k1 = sb;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j >= kb.n) break;
                const float4 kv = reinterpret_cast<const float4 *>((const float *)kb.p[j] + c * ns)[q];
                const float b = kb.af[j], e = ke.af[j];
                sb.x += b * kv.x; sb.y += b * kv.y; sb.z += b * kv.z; sb.w += b * kv.w;
                if (j == 0) {
                    k1 = kv;
                } else {
                    se.x += e * (kv.x - k1.x); se.y += e * (kv.y - k1.y);
                    se.z += e * (kv.z - k1.z); se.w += e * (kv.w - k1.w);
                }
            }
            const float4 m0 = reinterpret_cast<const float4 *>(mf + c * ns)[q];
            part.x += dp5_err_term(m0.x, sb.x, se.x, dtf, rtol, atol);
            part.y += dp5_err_term(m0.y, sb.y, se.y, dtf, rtol, atol);
            part.z += dp5_err_term(m0.z, sb.z, se.z, dtf, rtol, atol);
            part.w += dp5_err_term(m0.w, sb.w, se.w, dtf, rtol, atol);
        }
        const float s4 = (im.x > 0.f ? part.x : 0.f) + (im.y > 0.f ? part.y : 0.f) + (im.z > 0.f ? part.z : 0.f) +
                         (im.w > 0.f ? part.w : 0.f);
        acc += (double)s4;
    }
    if (blockIdx.x == 0 && threadIdx.x < (n_nodes & 3)) {
        const long n = 4 * n4 + threadIdx.x;
        float part = 0.f;
        for (int c = 0; c < 3; ++c) {
            const long i = c * ns + n;
            float sb = 0.f, se = 0.f, k1 = 0.f;
            for (int j = 0; j < 8; ++j) {
                if (j >= kb.n) break;
                const float kv = ((const float *)kb.p[j])[i];
                sb += kb.af[j] * kv;
                if (j == 0) k1 = kv;
                else se += ke.af[j] * (kv - k1);
            }
            part += dp5_err_term(mf[i], sb, se, dtf, rtol, atol);
        }
        if (inv_mass[n] > 0.f) acc += (double)part;
    }
    double s = block_sum<float>(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// One block: err = sqrt(sum partials / (3 n_active)); accept when err <= 1; new dt from
// dt * clamp(0.9 err^(-1/5), 0.2, 5); clipping to t_end; failure after too many rejections.
__global__ void __launch_bounds__(1024) k_dp5_ctl(const double *partials, int nparts, double n_active, StepCtl *ctl,
                                                  int max_rej)
{
    __shared__ double sh[1024];
    if (ctl->done) {
        if (threadIdx.x == 0) ctl->accepted = 0;
        return;
    }
    double v = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += partials[i];
    double s = block_sum<double>(v, sh);
    if (threadIdx.x != 0) return;
    double err = n_active > 0 ? sqrt(s / (3.0 * n_active)) : 0.0;
    bool fin = isfinite(err);
    bool acc = fin && err <= 1.0;
    double fac = !fin ? 0.2 : (err == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2))));
    ctl->err = err;
    ctl->accepted = acc;
    ctl->dt_used = ctl->dt;
    if (acc) {
        ctl->t += ctl->dt;
        ctl->n_acc += 1;
        ctl->consecutive_rej = 0;
    } else {
        ctl->n_rej += 1;
        ctl->consecutive_rej += 1;
    }
    double dtn = ctl->dt * fac;
    ctl->dt_prop = dtn;
    if (ctl->t_end > 0.0) {
        double rem = ctl->t_end - ctl->t;
        if (rem <= 1e-12 * fmax(fabs(ctl->t_end), 1e-30)) {
            ctl->done = 1;
        } else if (dtn > rem) {
            dtn = rem;
        }
    }
    if (ctl->consecutive_rej > max_rej || (!ctl->done && dtn < ctl->dt_min)) {
        ctl->status = NM_ERR_STEP_UNDERFLOW;
        ctl->done = 1;
    }
    ctl->dt = dtn;
}

// m + dt * sum_j b_j k_j, optionally renormalised (FP64 result; slope combination in the working
// precision, and in the FP32 path the norm through rsqrt_refined)
template <typename T>
__device__ __forceinline__ void advance_node(long n, long ns, const double *__restrict__ m, const KList &kb, double dt,
                                             int renorm, double v[3])
{
    for (int c = 0; c < 3; ++c) {
        long i = c * ns + n;
        T sb = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j >= kb.n) break;
            sb += kcoef<T>(kb, j) * ((const T *)kb.p[j])[i];
        }
        v[c] = m[i] + dt * (double)sb;
    }
    if (renorm) {
        const double s = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if (s > 0.0) {
            const double r = sizeof(T) == 8 ? 1.0 / sqrt(s) : rsqrt_refined(s);
            v[0] *= r; v[1] *= r; v[2] *= r;
        }
    }
}

// FP32 <-> FP64 conversions with integer operations, bit-identical to the hardware conversions in the
// normal range (float -> double is exact; double -> float rounds to nearest even).  Magnitudes below
// the smallest normal float (1.2e-38) become signed zeros; out-of-range values take the hardware path.
// The update of the FP32 path is bound by GB300's FP64 pipe, which would also carry the conversions.
__device__ __forceinline__ double f2d_int(float x)
{
    const unsigned u = __float_as_uint(x), a = u & 0x7fffffffu;
    if (a < 0x00800000u) return 0.0;
    if (a >= 0x7f800000u) return (double)x;
    const unsigned hi = (u & 0x80000000u) | ((a >> 3) + 0x38000000u);  // exponent bias 127 -> 1023
    return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ float d2f_int(double v)
{
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const unsigned ahi = hi & 0x7fffffffu, sign = hi & 0x80000000u, e = ahi >> 20;
    if (e <= 896u) return __uint_as_float(sign);
    if (e >= 1151u) return (float)v;
    unsigned f = ((e - 896u) << 23) | ((ahi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned r = lo & 0x1fffffffu;  // the 29 dropped mantissa bits
    f += (r > 0x10000000u || (r == 0x10000000u && (f & 1u))) ? 1u : 0u;  // a carry moves into the exponent
    return __uint_as_float(sign | f);
}

// v <- m + d (d = dt sum_j b_j k_j in FP32), optionally renormalised, and its FP32 copy.  FP64 work: the
// three additions, s = |v|^2 (three operations), e = s - 1, and v (1 + rho) with
//   rho = (1 + e)^(-1/2) - 1 = -e/2 + 3e^2/8 - 5e^3/16 + 35e^4/128 + O(e^5):
// the first term in FP64, the rest in FP32 (|e| < 1e-3: truncation below 3e-16, |v| - 1 below 1e-13).
// Larger e (a first step from a state that is not unit length) takes the refined reciprocal square root.
__device__ __forceinline__ void advance_f32(double v[3], const float d[3], int renorm, float f[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] += f2d_int(d[c]);
    if (renorm) {
        const double s = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if (s > 0.0) {
            const double e = s - 1.0;
            const float ef = d2f_int(e);
            if (fabsf(ef) < 1e-3f) {
                const double r = fma(-0.5, e, f2d_int(ef * ef * (0.375f + ef * (-0.3125f + ef * 0.2734375f))));
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] = fma(v[c], r, v[c]);
            } else {
                const double r = rsqrt_refined(s);
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] *= r;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] = d2f_int(v[c]);
}

// Accepted DP5 step of the FP32 path with the FP32 copy of m: four consecutive nodes per thread
// (16-byte slope loads, two 16-byte FP64 loads per component); the ragged tail node by node.
__global__ void k_dp5_update_f4(long n_nodes, long ns, double *__restrict__ m, KList kb, const float *__restrict__ k7,
                                float *__restrict__ k1, const StepCtl *ctl, int renorm, float *__restrict__ mf)
{
    const long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (!ctl->accepted) return;
    const float dtf = (float)ctl->dt_used;
    const long n4 = n_nodes >> 2;
    if (q < n4) {
        float d[3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 sb = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j >= kb.n) break;
                const float4 kv = reinterpret_cast<const float4 *>((const float *)kb.p[j] + c * ns)[q];
                const float b = kb.af[j];
                sb.x += b * kv.x; sb.y += b * kv.y; sb.z += b * kv.z; sb.w += b * kv.w;
            }
            d[c][0] = dtf * sb.x; d[c][1] = dtf * sb.y; d[c][2] = dtf * sb.z; d[c][3] = dtf * sb.w;
        }
        double v[3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 a = reinterpret_cast<const double2 *>(m + c * ns)[2 * q];
            const double2 b = reinterpret_cast<const double2 *>(m + c * ns)[2 * q + 1];
            v[c][0] = a.x; v[c][1] = a.y; v[c][2] = b.x; v[c][3] = b.y;
        }
        float f[3][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            double w[3] = {v[0][u], v[1][u], v[2][u]};
            const float dd[3] = {d[0][u], d[1][u], d[2][u]};
            float ff[3];
            advance_f32(w, dd, renorm, ff);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[c][u] = w[c];
                f[c][u] = ff[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            reinterpret_cast<double2 *>(m + c * ns)[2 * q] = make_double2(v[c][0], v[c][1]);
            reinterpret_cast<double2 *>(m + c * ns)[2 * q + 1] = make_double2(v[c][2], v[c][3]);
            reinterpret_cast<float4 *>(mf + c * ns)[q] = make_float4(f[c][0], f[c][1], f[c][2], f[c][3]);
            reinterpret_cast<float4 *>(k1 + c * ns)[q] = reinterpret_cast<const float4 *>(k7 + c * ns)[q];
        }
    }
    if (q < (n_nodes & 3)) {
        const long n = 4 * n4 + q;
        double w[3];
        float dd[3], ff[3];
        for (int c = 0; c < 3; ++c) {
            const long i = c * ns + n;
            float sb = 0.f;
            for (int j = 0; j < 8; ++j) {
                if (j >= kb.n) break;
                sb += kb.af[j] * ((const float *)kb.p[j])[i];
            }
            dd[c] = dtf * sb;
            w[c] = m[i];
        }
        advance_f32(w, dd, renorm, ff);
        for (int c = 0; c < 3; ++c) {
            const long i = c * ns + n;
            m[i] = w[c];
            mf[i] = ff[c];
            k1[i] = k7[i];
        }
    }
}

// Accepted step: m <- m5 (optionally renormalised), k1 <- k7 (FSAL).  Rejected: nothing.
template <typename T>
__global__ void k_dp5_update(long n_nodes, long ns, double *__restrict__ m, KList kb, const T *__restrict__ k7,
                             T *__restrict__ k1, const StepCtl *ctl, int renorm, float *__restrict__ mf)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    if (!ctl->accepted) return;
    double v[3];
    advance_node<T>(n, ns, m, kb, ctl->dt_used, renorm, v);
    for (int c = 0; c < 3; ++c) {
        long i = c * ns + n;
        m[i] = v[c];
        if (mf) mf[i] = (float)v[c];
        k1[i] = k7[i];
    }
}

// RK4 end of step: m <- m + dt/6 (k1 + 2 k2 + 2 k3 + k4), optional renormalisation.
template <typename T>
__global__ void k_rk4_update(long n_nodes, long ns, double *__restrict__ m, KList kb, const StepCtl *ctl, int renorm,
                             float *__restrict__ mf)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    if (ctl->done) return;
    double v[3];
    advance_node<T>(n, ns, m, kb, ctl->dt, renorm, v);
    for (int c = 0; c < 3; ++c) {
        m[c * ns + n] = v[c];
        if (mf) mf[c * ns + n] = (float)v[c];
    }
}

__global__ void k_rk4_advance(StepCtl *ctl)
{
    if (ctl->done) return;
    ctl->t += ctl->dt;
    ctl->n_acc += 1;
    ctl->accepted = 1;
    ctl->dt_used = ctl->dt;
    if (ctl->t_end > 0.0) {
        double rem = ctl->t_end - ctl->t;
        if (rem <= 1e-12 * fmax(fabs(ctl->t_end), 1e-30)) ctl->done = 1;
        else if (ctl->dt > rem) ctl->dt = rem;
    }
}

// Volume-weighted mean of m: per-block partial sums of (w m_x, w m_y, w m_z, w).
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_mean_partials(long n_nodes, long ns, const double *__restrict__ m,
                                                                const T *__restrict__ vol, double *partials)
{
    __shared__ double sh[kRedThreads];
    double a[4] = {0, 0, 0, 0};
    for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < n_nodes; n += (long)gridDim.x * blockDim.x) {
        double w = (double)vol[n];
        a[0] += w * m[n];
        a[1] += w * m[ns + n];
        a[2] += w * m[2 * ns + n];
        a[3] += w;
    }
    for (int c = 0; c < 4; ++c) {
        double s = block_sum<T>(a[c], sh);
        if (threadIdx.x == 0) partials[4 * blockIdx.x + c] = s;
    }
}

__global__ void __launch_bounds__(1024) k_mean_final(const double *partials, int nparts, double *out)
{
    __shared__ double sh[1024];
    for (int c = 0; c < 4; ++c) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += partials[4 * i + c];
        double s = block_sum<double>(v, sh);
        if (threadIdx.x == 0) sh[0] = s;
        if (threadIdx.x == 0) out[c] = s;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double w = out[3];
        for (int c = 0; c < 3; ++c) out[c] = w > 0 ? out[c] / w : 0.0;
    }
}

// Boundary layout (n1, n2, n3, comp) <-> internal SoA comp-planes with n1 fastest: a transpose of the
// n1 and n3 axes for each n2, through 32 x 32 shared-memory tiles so that both sides are accessed in
// contiguous runs (the boundary side may be page-locked host memory read or written over the
// host-device link).  Block (32, 8); grid (tiles along n3, tiles along n1, nn2).
constexpr int kTT = 32;
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) k_aos_to_soa(Geom g, const Tin *__restrict__ a, Tout *__restrict__ s,
                                                    unsigned long long *__restrict__ nonfinite)
{
    __shared__ Tout tile[3][kTT][kTT + 1];
    const int n2 = blockIdx.z;
    const int n3_0 = blockIdx.x * kTT, n1_0 = blockIdx.y * kTT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < kTT; r += 8) {
        const int n1 = n1_0 + r, n3 = n3_0 + tx;
        if (n1 < g.nn1 && n3 < g.nn3) {
            const long b = (((long)n1 * g.nn2 + n2) * g.nn3 + n3) * 3;
            const Tin v0 = a[b], v1 = a[b + 1], v2 = a[b + 2];
            if (nonfinite && !(isfinite(v0) && isfinite(v1) && isfinite(v2))) atomicAdd(nonfinite, 1ull);
            tile[0][r][tx] = (Tout)v0;
            tile[1][r][tx] = (Tout)v1;
            tile[2][r][tx] = (Tout)v2;
        }
    }
    __syncthreads();
    for (int r = ty; r < kTT; r += 8) {
        const int n3 = n3_0 + r, n1 = n1_0 + tx;
        if (n1 < g.nn1 && n3 < g.nn3) {
            const long n = ((long)n3 * g.nn2 + n2) * g.nn1 + n1;
            s[n] = tile[0][tx][r];
            s[g.ns + n] = tile[1][tx][r];
            s[2 * g.ns + n] = tile[2][tx][r];
        }
    }
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) k_soa_to_aos(Geom g, const Tin *__restrict__ s, Tout *__restrict__ a)
{
    __shared__ Tout tile[3][kTT][kTT + 1];
    const int n2 = blockIdx.z;
    const int n3_0 = blockIdx.x * kTT, n1_0 = blockIdx.y * kTT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < kTT; r += 8) {
        const int n3 = n3_0 + r, n1 = n1_0 + tx;
        if (n1 < g.nn1 && n3 < g.nn3) {
            const long n = ((long)n3 * g.nn2 + n2) * g.nn1 + n1;
            tile[0][tx][r] = (Tout)s[n];
            tile[1][tx][r] = (Tout)s[g.ns + n];
            tile[2][tx][r] = (Tout)s[2 * g.ns + n];
        }
    }
    __syncthreads();
    for (int r = ty; r < kTT; r += 8) {
        const int n1 = n1_0 + r, n3 = n3_0 + tx;
        if (n1 < g.nn1 && n3 < g.nn3) {
            const long b = (((long)n1 * g.nn2 + n2) * g.nn3 + n3) * 3;
            a[b] = tile[0][r][tx];
            a[b + 1] = tile[1][r][tx];
            a[b + 2] = tile[2][r][tx];
        }
    }
}

// Cell fields: boundary (c1, c2, c3[, comp]) -> internal c1-fastest (SoA planes for vectors).
template <typename Tout>
__global__ void k_cells_to_internal(Geom g, const double *__restrict__ a, int ncomp, double scale_by_Ms0,
                                    const double *__restrict__ Ms, Tout *__restrict__ s)
{
    long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (c >= g.n_cells) return;
    const int c1 = (int)(c % g.N1);
    const long r = c / g.N1;
    const int c2 = (int)(r % g.N2);
    const int c3 = (int)(r / g.N2);
    long b = (((long)c1 * g.N2 + c2) * g.N3 + c3) * ncomp;
    double f = scale_by_Ms0 != 0.0 ? (Ms ? Ms[c] : scale_by_Ms0) : 1.0;
    for (int j = 0; j < ncomp; ++j) s[j * g.cs + c] = (Tout)(f * a[b + j]);
}

template <typename Tin, typename Tout>
__global__ void k_convert(long n, const Tin *__restrict__ a, Tout *__restrict__ b)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (Tout)a[i];
}

// volume weights of the nodal mean: sum over adjacent magnetic cells of V/8 (V/4 per in-plane cell and
// layer with the 2D basis, V/2 per cell of the two slabs beside the node with the 1D basis)
template <typename T>
__global__ void k_node_volume(Geom g, const double *__restrict__ Ms, double Ms0, double V8, T *vol)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= g.n_nodes) return;
    const int n1 = (int)(n % g.nn1);
    const long r = n / g.nn1;
    const int n2 = (int)(r % g.nn2);
    const int n3 = (int)(r / g.nn2);
    double s = 0.0;
    if (g.basis == 2) {  // 2D basis: the 4 in-plane cells of every layer, V/4 each
        for (int i = 0; i < 4; ++i) {
            const int c1 = n1 - ((i >> 1) & 1), c2 = n2 - (i & 1);
            if (c1 < 0 || c1 >= g.N1 || c2 < 0 || c2 >= g.N2) continue;
            for (int c3 = 0; c3 < g.N3; ++c3)
                if ((Ms ? Ms[((long)c3 * g.N2 + c2) * g.N1 + c1] : Ms0) > 0.0) s += 2.0 * V8;
        }
    } else if (g.basis == 1) {  // 1D basis: every cell of the two slabs beside the node, V/2 each
        for (int c1 = n1 - 1; c1 <= n1; ++c1) {
            if (c1 < 0 || c1 >= g.N1) continue;
            for (long j = 0; j < (long)g.N2 * g.N3; ++j)
                if ((Ms ? Ms[j * g.N1 + c1] : Ms0) > 0.0) s += 4.0 * V8;
        }
    } else {
        for (int i = 0; i < 8; ++i) {
            int c1 = n1 - ((i >> 2) & 1), c2 = n2 - ((i >> 1) & 1), c3 = n3 - (i & 1);
            if (c1 >= 0 && c1 < g.N1 && c2 >= 0 && c2 < g.N2 && c3 >= 0 && c3 < g.N3) {
                double ms = Ms ? Ms[((long)c3 * g.N2 + c2) * g.N1 + c1] : Ms0;
                if (ms > 0.0) s += V8;
            }
        }
    }
    vol[n] = (T)s;
}

// ---------------------------------------------------------------------------------------------
// the list with its FP32 coefficients filled in
static KList fk(const KList &k)
{
    KList r = k;
    for (int j = 0; j < 8; ++j) r.af[j] = (float)k.a[j];
    return r;
}

template <typename T>
void launch_stage_input(const Geom &g, const double *m, const KList &k, const StepCtl *ctl, T *y, cudaStream_t st,
                        const float *mf)
{
    if constexpr (sizeof(T) == 4) {
        if (mf) {
            const long n4 = g.n_nodes >> 2;
            k_stage_input_f4<<<div_up(n4 > 4 ? n4 : 4, 256), 256, 0, st>>>(g.n_nodes, g.ns, fk(k), ctl, (float *)y, mf);
            return;
        }
    }
    k_stage_input<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g.n_nodes, g.ns, m, fk(k), ctl, y, mf);
}

int reduction_blocks(long n_nodes)
{
    long b = (n_nodes + kRedThreads - 1) / kRedThreads;
    return (int)(b > 1024 ? 1024 : (b < 1 ? 1 : b));
}

template <typename T>
void launch_dp5_control(const Geom &g, const double *m, const KList &kb, const KList &ke, const T *inv_mass,
                        StepCtl *ctl, double *partials, double n_active, int max_rej, cudaStream_t st,
                        const float *mf, bool f64_terms)
{
    // up to 4096 partial sums (the mesh's partials buffer), so that enough loads are in flight
    long nbl = (g.n_nodes + kRedThreads - 1) / kRedThreads;
    const int nb = (int)(nbl > 4096 ? 4096 : (nbl < 1 ? 1 : nbl));
    if constexpr (sizeof(T) == 4) {
        if (f64_terms) {
            k_dp5_err<T, true><<<nb, kRedThreads, 0, st>>>(g.n_nodes, g.ns, m, fk(kb), fk(ke), inv_mass, ctl,
                                                           partials, nullptr);
            k_dp5_ctl<<<1, 1024, 0, st>>>(partials, nb, n_active, ctl, max_rej);
            return;
        }
        if (mf) {
            k_dp5_err_f4<<<nb, kRedThreads, 0, st>>>(g.n_nodes, g.ns, fk(kb), fk(ke), (const float *)inv_mass, ctl,
                                                     partials, mf);
            k_dp5_ctl<<<1, 1024, 0, st>>>(partials, nb, n_active, ctl, max_rej);
            return;
        }
    }
    k_dp5_err<T><<<nb, kRedThreads, 0, st>>>(g.n_nodes, g.ns, m, fk(kb), fk(ke), inv_mass, ctl, partials, mf);
    k_dp5_ctl<<<1, 1024, 0, st>>>(partials, nb, n_active, ctl, max_rej);
}

template <typename T>
void launch_dp5_update(const Geom &g, double *m, const KList &kb, const T *k7, T *k1, const StepCtl *ctl, int renorm,
                       cudaStream_t st, float *mf)
{
    if constexpr (sizeof(T) == 4) {
        if (mf) {
            const long n4 = g.n_nodes >> 2;
            k_dp5_update_f4<<<div_up(n4 > 4 ? n4 : 4, 256), 256, 0, st>>>(g.n_nodes, g.ns, m, fk(kb), (const float *)k7,
                                                                           (float *)k1, ctl, renorm, mf);
            return;
        }
    }
    k_dp5_update<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g.n_nodes, g.ns, m, fk(kb), k7, k1, ctl, renorm, mf);
}

template <typename T>
void launch_rk4_update(const Geom &g, double *m, const KList &kb, StepCtl *ctl, int renorm, cudaStream_t st,
                       float *mf)
{
    k_rk4_update<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g.n_nodes, g.ns, m, fk(kb), ctl, renorm, mf);
    k_rk4_advance<<<1, 1, 0, st>>>(ctl);
}

template <typename T>
void launch_mean(const Geom &g, const double *m, const T *vol, double *partials, double *out, cudaStream_t st)
{
    int nb = reduction_blocks(g.n_nodes);
    k_mean_partials<T><<<nb, kRedThreads, 0, st>>>(g.n_nodes, g.ns, m, vol, partials);
    k_mean_final<<<1, 1024, 0, st>>>(partials, nb, out);
}

template <typename Tin, typename Tout>
void launch_aos_to_soa(const Geom &g, const Tin *a, Tout *s, cudaStream_t st, unsigned long long *nonfinite)
{
    const dim3 grid(div_up(g.nn3, kTT), div_up(g.nn1, kTT), g.nn2);
    k_aos_to_soa<Tin, Tout><<<grid, dim3(kTT, 8), 0, st>>>(g, a, s, nonfinite);
}

template <typename Tin, typename Tout>
void launch_soa_to_aos(const Geom &g, const Tin *s, Tout *a, cudaStream_t st)
{
    const dim3 grid(div_up(g.nn3, kTT), div_up(g.nn1, kTT), g.nn2);
    k_soa_to_aos<Tin, Tout><<<grid, dim3(kTT, 8), 0, st>>>(g, s, a);
}

template <typename Tout>
void launch_cells_to_internal(const Geom &g, const double *a, int ncomp, double scale_by_Ms0, const double *Ms,
                              Tout *s, cudaStream_t st)
{
    k_cells_to_internal<Tout><<<div_up(g.n_cells, 256), 256, 0, st>>>(g, a, ncomp, scale_by_Ms0, Ms, s);
}

template <typename Tin, typename Tout>
void launch_convert(long n, const Tin *a, Tout *b, cudaStream_t st)
{
    k_convert<Tin, Tout><<<div_up(n, 256), 256, 0, st>>>(n, a, b);
}

template <typename T>
void launch_node_volume(const Geom &g, const double *Ms, double Ms0, double V, T *vol, cudaStream_t st)
{
    k_node_volume<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g, Ms, Ms0, V / 8.0, vol);
}

#define NM_INST(T)                                                                                             \
    template void launch_stage_input<T>(const Geom &, const double *, const KList &, const StepCtl *, T *,       \
                                        cudaStream_t, const float *);                                                         \
    template void launch_dp5_control<T>(const Geom &, const double *, const KList &, const KList &, const T *,   \
                                        StepCtl *, double *, double, int, cudaStream_t, const float *, bool);                 \
    template void launch_dp5_update<T>(const Geom &, double *, const KList &, const T *, T *, const StepCtl *,  \
                                       int, cudaStream_t, float *);                                                     \
    template void launch_rk4_update<T>(const Geom &, double *, const KList &, StepCtl *, int, cudaStream_t, float *);    \
    template void launch_mean<T>(const Geom &, const double *, const T *, double *, double *, cudaStream_t);     \
    template void launch_cells_to_internal<T>(const Geom &, const double *, int, double, const double *, T *,  \
                                              cudaStream_t);                                                   \
    template void launch_node_volume<T>(const Geom &, const double *, double, double, T *, cudaStream_t);

NM_INST(float)
NM_INST(double)
template void launch_aos_to_soa<float, float>(const Geom &, const float *, float *, cudaStream_t,
                                              unsigned long long *);
template void launch_aos_to_soa<double, float>(const Geom &, const double *, float *, cudaStream_t,
                                               unsigned long long *);
template void launch_aos_to_soa<double, double>(const Geom &, const double *, double *, cudaStream_t,
                                                unsigned long long *);
template void launch_soa_to_aos<float, float>(const Geom &, const float *, float *, cudaStream_t);
template void launch_soa_to_aos<float, double>(const Geom &, const float *, double *, cudaStream_t);
template void launch_soa_to_aos<double, double>(const Geom &, const double *, double *, cudaStream_t);
template void launch_convert<double, float>(long, const double *, float *, cudaStream_t);
template void launch_convert<double, double>(long, const double *, double *, cudaStream_t);
template void launch_convert<float, double>(long, const float *, double *, cudaStream_t);

}  // namespace nm
