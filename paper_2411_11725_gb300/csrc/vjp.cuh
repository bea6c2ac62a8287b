// Kernels of the transposed (adjoint) products of the effective field and of the LLG right-hand side.
#pragma once
#include "local.cuh"

namespace nm {

// w = v * (1/mass) per node (0 where no magnetic cell touches the node)
template <typename T>
void launch_scale_inv_mass(const Geom &g, const T *v, const T *inv_mass, T *w, cudaStream_t st);

// out_c = Ms_c * scale * sum_{i in {0,1}^3} y_{c+i} per cell and component (scale 1/8: cell mean)
template <typename T>
void launch_cell_moment(const Geom &g, const T *y, const T *Ms, T Ms0, T scale, T *out, cudaStream_t st);

// Gradient of <v, h(m)> with respect to the cell Ms map (accumulated into gMs, FP64, cell layout c1
// fastest):
//   mu0 V/8 [ W_c . (H_c + s_c h_c) + m_c . HW_c - sum_{n in c} w_n . (h_n - h_u) ]
// with w = v / mass, W_c = sum of w over the 8 corners, m_c the corner mean of m, H the demag cell
// field of Ms m_c, HW that of Ms W_c, h the effective field at m and h_u the uniform applied field.
struct GradMsArgs {
    const void *m, *w, *h, *H, *HW;  // working precision
    const double *hcell;               // cell applied field (3 x cs) or NULL
    double sc;                         // its time factor
    double hu[3];                      // uniform applied field at t (A/m)
    double mu0V8;
    int demag;                         // include the demag parts
    double weight;                     // gMs += weight * gradient
};
template <typename T>
void launch_grad_Ms(const Geom &g, const GradMsArgs &a, const T *inv_mass, double *gMs, cudaStream_t st);

// LLG transpose product, local part.  With f(y) = -g'(y x H + alpha y x (y x H)) and cotangent u:
//   ybar_local = -g'[ H x u + alpha ((y x H) x u + H x (u x y)) ]
//   q          = -g'[ u x y + alpha (u x y) x y ]          (cotangent of H, fed to the h_eff VJP)
// zero on nodes without magnetic material.  ybar_local is written to ybar (accumulated with `acc`).
template <typename T>
void launch_llg_vjp_local(const Geom &g, const T *y, const T *H, const T *u, const T *inv_mass, double gam,
                          double alpha, T *ybar, T *q, cudaStream_t st);

// out = a * x + b * y (nodal SoA, 3 components)
template <typename T>
void launch_axpby(const Geom &g, T a, const T *x, T b, const T *y, T *out, cudaStream_t st);

}  // namespace nm

namespace nm {
// internal cell layout (c1 fastest, FP64) -> boundary cell layout (c1 slowest) in type To
template <typename To>
void launch_cells_to_boundary(const Geom &g, const double *s, To *a, cudaStream_t st);
}  // namespace nm

namespace nm {

// Weighted sums over nodal SoA buffers; sources in the working precision (pt) or in FP64 (pd).
struct LinComb {
    const void *pt[8];
    double at[8];
    int nt;
    const double *pd[2];
    double ad[2];
    int nd;
};
// out (working precision) = sum_j at_j pt_j + sum_j ad_j pd_j
template <typename T>
void launch_lincomb(const Geom &g, const LinComb &lc, T *out, cudaStream_t st);
// out (FP64) = sum_j at_j pt_j + sum_j ad_j pd_j
template <typename T>
void launch_lincomb_d(const Geom &g, const LinComb &lc, double *out, cudaStream_t st);

// Adjoint of the end of a step, m_next = N(mt), mt = m + dt sum_j b_j k_j, N(x) = x/|x| when renorm:
//   lam_t = (lam - (mh . lam) mh) / |mt|   (mh = mt/|mt|),   or lam_t = lam without renormalisation.
// Writes lam_t in FP64 and in the working precision.
template <typename T>
void launch_renorm_adjoint(const Geom &g, const double *m, const LinComb &kb, double dt, const double *lam,
                           int renorm, double *lam_t, T *lam_t_w, cudaStream_t st);

// Sampled quadratic loss at one time: partial sums of sum W (m - target)^2 per block, and
// lam += 2 W (m - target) when lam != NULL.  `target` may be NULL (zero).  Returns the block count.
int launch_loss_terms(const Geom &g, const double *m, const double *W, const double *target, double *lam,
                      double *partials, cudaStream_t st);
// sum of the first n partials into out[0] (one block, fixed order)
void launch_sum_partials(const double *partials, int n, double *out, cudaStream_t st);

// acc[c][n] += scale * q[c][n] (FP64 nodal accumulator of a uniform-field gradient)
template <typename T>
void launch_accum_nodal(const Geom &g, const T *q, double scale, double *acc, cudaStream_t st);
// out[c] = sum_n acc[c][n] (deterministic two-level reduction through partials[3 x 1024])
void launch_sum_nodal3(const Geom &g, const double *acc, double *partials, double *out, cudaStream_t st);

}  // namespace nm
