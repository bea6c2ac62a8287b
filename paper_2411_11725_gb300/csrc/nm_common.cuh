// Shared definitions of the sm_103a library: complex arithmetic, mesh state, launch helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "nmgb.h"

namespace nm {

constexpr double kMu0 = 4.0e-7 * 3.14159265358979323846;

template <typename T> struct Cx;
template <> struct alignas(8) Cx<float> { float x, y; };
template <> struct alignas(16) Cx<double> { double x, y; };

template <typename T> __host__ __device__ __forceinline__ Cx<T> cx(T a, T b) { Cx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __host__ __device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return cx<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return cx<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ Cx<T> operator*(Cx<T> a, Cx<T> b)
{
    return cx<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ Cx<T> scale(Cx<T> a, T s) { return cx<T>(a.x * s, a.y * s); }
template <typename T> __host__ __device__ __forceinline__ Cx<T> conj(Cx<T> a) { return cx<T>(a.x, -a.y); }
// multiply by s*i for s = +-1
template <typename T> __host__ __device__ __forceinline__ Cx<T> mul_si(Cx<T> a, int s)
{
    return s > 0 ? cx<T>(-a.y, a.x) : cx<T>(a.y, -a.x);
}

// Division by a run-time constant through a multiply-high (round-up method): valid for n + d < 2^32.
struct FastDiv {
    unsigned d, m, s;
    FastDiv() = default;
    __host__ __device__ explicit FastDiv(unsigned d_) : d(d_), m(0), s(0)
    {
        while ((1u << s) < d) ++s;
        m = (unsigned)(((1ull << 32) * ((1ull << s) - d)) / d + 1);
    }
    __device__ __forceinline__ unsigned div(unsigned n) const { return (__umulhi(n, m) + n) >> s; }
    __device__ __forceinline__ unsigned mod(unsigned n) const { return n - div(n) * d; }
};

// Device-resident step control: every kernel of an RK step reads t and dt from here, so a whole step
// (or many) can be launched without a host round trip.
struct StepCtl {
    double t;        // time at the start of the step being attempted
    double dt;       // size of the step being attempted
    double dt_used;  // size of the last attempted step (read by the update after control)
    double dt_prop;  // controller proposal before clipping to t_end
    double err;      // error norm of the last attempt
    double t_end;    // integration end (run_until); steps are clipped to it and to sample times
    double sample_dt;
    double dt_min;
    long n_acc, n_rej;
    long next_sample;  // index of the next sample time (run_until)
    long max_samples;
    int accepted;    // last attempt accepted
    int done;        // t reached t_end: later steps do nothing
    int status;      // NM_OK or an NM_ERR_* code set on the device
    int consecutive_rej;
    double rtol, atol;
};

// Optional per-launch hook, called after every kernel launch with the kernel's name (profiling).
struct Marker {
    void (*fn)(void *ctx, const char *name) = nullptr;
    void *ctx = nullptr;
    void operator()(const char *name) const
    {
        if (fn) fn(ctx, name);
    }
};

// Launch-shape helpers
inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }
inline long round_up(long a, long b) { return (a + b - 1) / b * b; }

}  // namespace nm
