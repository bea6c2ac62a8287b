// Runge-Kutta bookkeeping kernels (stage inputs, error norm, step control, updates) and layout
// conversions.
#pragma once
#include "demag.cuh"

namespace nm {

// A weighted list of slope buffers: sum_j a[j] * p[j]
struct KList {
    const void *p[8];
    double a[8];
    int n;
    float af[8];  // a in FP32 (filled by the launch functions; used by the FP32 path)
};

// coefficient j of a slope list in the working precision
template <typename T>
__device__ __forceinline__ T kcoef(const KList &k, int j)
{
    if constexpr (sizeof(T) == 4) return k.af[j];
    else return (T)k.a[j];
}

int reduction_blocks(long n_nodes);

// mf: FP32 copy of m (FP32 path; NULL = use m).  Stage inputs and the error scale read it; the updates
// keep it equal to fl32(m).
template <typename T>
void launch_stage_input(const Geom &g, const double *m, const KList &k, const StepCtl *ctl, T *y, cudaStream_t st,
                        const float *mf = nullptr);
template <typename T>
// f64_terms (FP32 slopes): every per-node term of the error norm in FP64 instead of FP32
void launch_dp5_control(const Geom &g, const double *m, const KList &kb, const KList &ke, const T *inv_mass,
                        StepCtl *ctl, double *partials, double n_active, int max_rej, cudaStream_t st,
                        const float *mf = nullptr, bool f64_terms = false);
template <typename T>
void launch_dp5_update(const Geom &g, double *m, const KList &kb, const T *k7, T *k1, const StepCtl *ctl, int renorm,
                       cudaStream_t st, float *mf = nullptr);
template <typename T>
void launch_rk4_update(const Geom &g, double *m, const KList &kb, StepCtl *ctl, int renorm, cudaStream_t st,
                       float *mf = nullptr);
template <typename T>
void launch_mean(const Geom &g, const double *m, const T *vol, double *partials, double *out, cudaStream_t st);
template <typename Tin, typename Tout>
// node-major (n1, n2, n3, 3) -> SoA planes; with `nonfinite` set, also counts the nodes holding a
// non-finite component into *nonfinite (device)
void launch_aos_to_soa(const Geom &g, const Tin *a, Tout *s, cudaStream_t st, unsigned long long *nonfinite = nullptr);
template <typename Tin, typename Tout>
void launch_soa_to_aos(const Geom &g, const Tin *s, Tout *a, cudaStream_t st);
template <typename Tout>
void launch_cells_to_internal(const Geom &g, const double *a, int ncomp, double scale_by_Ms0, const double *Ms,
                              Tout *s, cudaStream_t st);
template <typename Tin, typename Tout>
void launch_convert(long n, const Tin *a, Tout *b, cudaStream_t st);
template <typename T>
void launch_node_volume(const Geom &g, const double *Ms, double Ms0, double V, T *vol, cudaStream_t st);

}  // namespace nm
