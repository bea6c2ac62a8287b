// Local field terms and the LLG right-hand side, fused per node.
#pragma once
#include "demag.cuh"

namespace nm {

// Per-mesh constants of the local terms.  The cell-local exchange and consistent-mass integrals of
// the trilinear basis depend only on d = |i - i'| per direction (bit 2: direction 1, bit 1:
// direction 2, bit 0: direction 3), so 8 numbers per term describe the 24x24 element matrices.
template <typename T>
struct LocalParams {
    Geom g;
    T Wex[8];          // int_cell 2 grad(phi_i).grad(phi_i') for the pattern d (per unit A)
    T Wm[8];           // int_cell phi_i phi_i' for the pattern d
    // Interior nodes of a uniform material (no cell maps, Ms0 > 0): the 27 assembled weights of the
    // neighbour offsets o (index (o3+1)*9 + (o2+1)*3 + (o1+1)), exchange (self weight unused) and
    // anisotropy, and the sum of the exchange weights.  uniform = 0 disables that path.
    int uniform;
    T wex27[27], wan27[27], wex_sum;
    // uniform material at any node: Wex[d] A and Wm[d] Ku (0 for terms that are off); the weight of an
    // offset is this times the number of mesh cells that hold both nodes, a product of per-axis counts
    T wexd[8], wand[8];
    T mu0V8;           // mu0 * V / 8
    // 2D basis (section "Low-Dimensional Geometries"): the in-plane pattern integrals per cell layer
    // (pattern d = 2 |o1| + |o2|), through the layer's thickness, and mu0 V / 4
    T Wex2[4], Wm2[4], mu0V4;
    // interfacial DMI: raw field buffer (NULL: term off), cell map or uniform value, and the pattern
    // weights of the antisymmetric element integrals (dmx by (|o2|,|o3|), dmy by (|o1|,|o3|))
    T *hdmi;
    const T *Dm;
    T D0, dmx[4], dmy[4];
    const T *A;        // cell maps (n_cells) or NULL for the uniform value
    const T *Ku;
    const T *Ms;
    T A0, Ku0, Ms0;
    T e0, e1, e2;      // easy axis
    const T *inv_mass; // 1/mass_n, 0 where no magnetic cell touches n
    const T *MsH;      // demag: Ms_c H_c (3 x cs) or NULL
    const T *Msh;      // cell applied field times Ms: Ms_c h_c (3 x cs) or NULL
    double hu0, hu1, hu2, hu_freq, hu_phase, hc_freq, hc_phase;
    unsigned terms;
    double gam;        // gamma / (1 + alpha^2)
    T gam_t, alpha_t;  // the same in the working precision
    int raw;           // 1: output -dE (no division by the mass, no uniform applied field)
    double alpha;
    // 1D basis: the pattern integrals along x (d = |o1|) per cell of the cross-section, through its
    // area, and mu0 V / 2 (last, so that the fields above keep the offsets the other kernels were tuned
    // with)
    T Wex1[2], Wm1[2], mu0V2;
};

// What the node kernel writes.
//   out_h:   H (3 x ns) -- effective-field evaluation
//   k_out:   LLG slope k_s (3 x ns)
//   y_next:  next stage input y_{s+1} = m + dt sum_{j<=s} a_j k_j (3 x ns), when non-NULL
struct StageArgs {
    const double *m;          // FP64 master magnetisation (3 x ns)
    const float *mf;          // its FP32 copy (FP32 path; NULL = form the next input from m in FP64)
    const void *k[8];         // k_1 .. k_s (k[s-1] is the one being written)
    double a[8];              // a_{s+1, j}, j = 1 .. s
    int s;                    // stage index (1-based) of the slope being computed
    double c_s;               // time fraction of stage s
    float af[8];              // the same coefficients in FP32 (used by the FP32 path)
    double a_s;               // a_{s+1, s}: the coefficient of the slope being written (a[s - 1])
    float af_s;
    const StepCtl *ctl;       // t, dt
    double t_fixed;           // time when ctl == NULL
};

template <typename T>
void launch_heff(const LocalParams<T> &p, const T *y, T *h_out, double t, cudaStream_t st);

template <typename T>
void launch_llg_stage(const LocalParams<T> &p, const T *y, T *k_out, T *y_next, const StageArgs &sa,
                      cudaStream_t st);

// lumped mass: inv_mass_n = 1 / (mu0 V/8 sum_{c∋n} Ms_c); counts magnetic nodes into *n_active (device)
template <typename T>
void launch_mass(const Geom &g, const double *Ms_d, double Ms0, double V, T *inv_mass, unsigned long long *n_active,
                 cudaStream_t st);

}  // namespace nm
