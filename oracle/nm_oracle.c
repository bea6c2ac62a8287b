/*
 * nm_oracle.c -- the FP64 CPU oracle for the nodal finite-difference effective field and LLG
 * integration of NeuralMag (arXiv 2411.11725).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file; only the
 * tests, the smoke check and the bench's CPU-baseline leg do.  It shares no code with the CUDA
 * library: it is written from the paper's definitions, in the paper's order, as plainly as possible.
 *
 *   - Nodal basis and element integrals by 2x2x2 Gauss quadrature of the trilinear reference basis
 *     (Sec. "Local Field Terms", Eq. nodal_basis and the reference basis below it).
 *   - Local terms by per-cell assembly of the cell-wise variation, n = c + i
 *     (Eqs. weak_form_impl_f_cell, weak_form_impl_f, weak_form_impl), with cell-wise material
 *     (Eqs. ms_discrete, cell_basis) and mass lumping (Eq. mass_lumping).
 *   - Demagnetisation field by the standard cuboid-cell FD method with node->cell and cell->node
 *     averaging (Sec. "Demagnetization Field"), evaluated as a DIRECT O(N^2) sum over cells.  The
 *     Newell tensor is evaluated in _Float128 so that its far-field cancellation does not limit
 *     FP64 parity.
 *   - LLG right-hand side (Eq. llg), classical RK4 and Dormand-Prince 5(4) (Sec. "Automatic
 *     Differentiation and Time Integration").
 *
 * Layouts (all FP64, C order): nodal vector fields (N1+1, N2+1, N3+1, 3); cell scalars (N1, N2, N3);
 * cell vectors (N1, N2, N3, 3).  SI units: m, A/m, J/m, J/m^3, s.
 *
 * Parity unpinned: gamma and the config-specific physical choices are conventions passed in by the
 * caller, not derived from the paper.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define MU0 (4.0e-7 * M_PI)

#define TERM_EXCH 1u
#define TERM_ANIS 2u
#define TERM_ZEE 4u
#define TERM_DEMAG 8u
#define TERM_DMI 16u

typedef _Float128 q128;

typedef struct {
    int N[3];
    double dx[3];
    double *Ms, *A, *Ku;          /* cells */
    double axis[3];
    double alpha, gamma;
    double hu[3], hu_freq, hu_phase;          /* uniform applied field, A/m */
    double *hcell, hc_freq, hc_phase;         /* optional cell-wise applied field (cells x 3) */
    double *Nt;                               /* demag tensor octant: (N1, N2, N3, 6), or NULL */
    double Kex[8][8];                         /* int_cell 2 grad(phi_i).grad(phi_i') */
    double Mm[8][8];                          /* int_cell phi_i phi_i' */
    double Phi[8];                            /* int_cell phi_i */
    double *D;                                /* interfacial DMI constant per cell (J/m^2) */
    double Gd[2][8][8];                       /* int_cell phi_i d_k phi_i', k = x, y */
} OrMesh;

/* ------------------------------------------------------------------------------------------------
 * Reference basis (Eq. nodal_basis and the definition of phi-hat below it):
 *   phi_i(xi) = prod_k [1 - i_k + (2 i_k xi_k - xi_k)],  xi in [0,1]^3, i in {0,1}^3.
 * Local vertex i = (i1,i2,i3) is numbered li = 4*i1 + 2*i2 + i3.
 * ---------------------------------------------------------------------------------------------- */
static double phi_1d(int i, double xi) { return 1.0 - i + (2.0 * i * xi - xi); }
static double dphi_1d(int i) { return 2.0 * i - 1.0; } /* d/dxi of phi_1d */

static void vertex_of(int li, int i[3]) { i[0] = (li >> 2) & 1; i[1] = (li >> 1) & 1; i[2] = li & 1; }

double or_phi(int li, double x1, double x2, double x3)
{
    int i[3];
    vertex_of(li, i);
    return phi_1d(i[0], x1) * phi_1d(i[1], x2) * phi_1d(i[2], x3);
}

/* physical gradient of the basis function of local vertex li at reference point xi */
static void grad_phi(int li, const double xi[3], const double dx[3], double g[3])
{
    int i[3];
    vertex_of(li, i);
    for (int k = 0; k < 3; ++k) {
        double v = dphi_1d(i[k]) / dx[k];
        for (int l = 0; l < 3; ++l)
            if (l != k) v *= phi_1d(i[l], xi[l]);
        g[k] = v;
    }
}

/* 2-point Gauss-Legendre rule on [0,1] in each direction: exact for the trilinear integrands here */
static void gauss_point(int q, double xi[3], double *w)
{
    const double a = 0.5 - 0.5 / sqrt(3.0), b = 0.5 + 0.5 / sqrt(3.0);
    xi[0] = (q & 4) ? b : a;
    xi[1] = (q & 2) ? b : a;
    xi[2] = (q & 1) ? b : a;
    *w = 0.125;
}

/* Element integrals of one cell (the 24x24 element matrix of Eq. weak_form_impl_f_cell is
 * block-diagonal in the component index for these isotropic terms, so the 8x8 blocks suffice). */
void or_element_matrices(double dx1, double dx2, double dx3, double *Kex, double *Mm, double *Phi)
{
    const double dx[3] = {dx1, dx2, dx3};
    const double V = dx1 * dx2 * dx3;
    for (int a = 0; a < 64; ++a) { Kex[a] = 0.0; Mm[a] = 0.0; }
    for (int a = 0; a < 8; ++a) Phi[a] = 0.0;
    for (int q = 0; q < 8; ++q) {
        double xi[3], w;
        gauss_point(q, xi, &w);
        for (int li = 0; li < 8; ++li) {
            double gi[3];
            grad_phi(li, xi, dx, gi);
            double pi = or_phi(li, xi[0], xi[1], xi[2]);
            Phi[li] += w * V * pi;
            for (int lj = 0; lj < 8; ++lj) {
                double gj[3];
                grad_phi(lj, xi, dx, gj);
                double pj = or_phi(lj, xi[0], xi[1], xi[2]);
                Kex[li * 8 + lj] += w * V * 2.0 * (gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2]);
                Mm[li * 8 + lj] += w * V * pi * pj;
            }
        }
    }
}

/* ------------------------------------------------------------------------------------------------
 * Index helpers
 * ---------------------------------------------------------------------------------------------- */
static long nidx(const OrMesh *o, int n1, int n2, int n3)
{
    return ((long)n1 * (o->N[1] + 1) + n2) * (o->N[2] + 1) + n3;
}
static long cidx(const OrMesh *o, int c1, int c2, int c3)
{
    return ((long)c1 * o->N[1] + c2) * o->N[2] + c3;
}
static long n_nodes(const OrMesh *o) { return (long)(o->N[0] + 1) * (o->N[1] + 1) * (o->N[2] + 1); }
static long n_cells(const OrMesh *o) { return (long)o->N[0] * o->N[1] * o->N[2]; }

/* ------------------------------------------------------------------------------------------------
 * Mesh object
 * ---------------------------------------------------------------------------------------------- */
void *or_create(int n1, int n2, int n3, double dx1, double dx2, double dx3)
{
    if (n1 < 1 || n2 < 1 || n3 < 1 || !(dx1 > 0) || !(dx2 > 0) || !(dx3 > 0)) return NULL;
    OrMesh *o = (OrMesh *)calloc(1, sizeof(OrMesh));
    o->N[0] = n1; o->N[1] = n2; o->N[2] = n3;
    o->dx[0] = dx1; o->dx[1] = dx2; o->dx[2] = dx3;
    long nc = n_cells(o);
    o->Ms = (double *)calloc(nc, sizeof(double));
    o->A = (double *)calloc(nc, sizeof(double));
    o->Ku = (double *)calloc(nc, sizeof(double));
    o->axis[2] = 1.0;
    o->alpha = 0.0;
    o->gamma = 0.0;
    or_element_matrices(dx1, dx2, dx3, &o->Kex[0][0], &o->Mm[0][0], o->Phi);
    o->D = (double *)calloc(nc, sizeof(double));
    {
        const double V = dx1 * dx2 * dx3;
        for (int q = 0; q < 8; ++q) {
            double xi[3], w;
            gauss_point(q, xi, &w);
            for (int li = 0; li < 8; ++li)
                for (int lj = 0; lj < 8; ++lj) {
                    double gj[3];
                    grad_phi(lj, xi, o->dx, gj);
                    const double pi = or_phi(li, xi[0], xi[1], xi[2]);
                    for (int k = 0; k < 2; ++k) o->Gd[k][li][lj] += w * V * pi * gj[k];
                }
        }
    }
    return o;
}

/* Interfacial Dzyaloshinskii-Moriya constant per cell (J/m^2); the energy is the reading
 *   E = int D [m_z div m - (m . grad) m_z]  (interface normal along z). */
void or_set_dmi(void *h, const double *D)
{
    OrMesh *o = (OrMesh *)h;
    memcpy(o->D, D, n_cells(o) * sizeof(double));
}

void or_free(void *h)
{
    OrMesh *o = (OrMesh *)h;
    if (!o) return;
    free(o->Ms); free(o->A); free(o->Ku); free(o->hcell); free(o->Nt); free(o->D);
    free(o);
}

/* Material (Eq. ms_discrete: cell-wise constants).  A cell with Ms = 0 is vacuum and contributes to
 * no term. */
void or_set_material(void *h, const double *Ms, const double *A, const double *Ku, const double *axis,
                     double alpha, double gamma)
{
    OrMesh *o = (OrMesh *)h;
    long nc = n_cells(o);
    memcpy(o->Ms, Ms, nc * sizeof(double));
    memcpy(o->A, A, nc * sizeof(double));
    memcpy(o->Ku, Ku, nc * sizeof(double));
    double n = sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    for (int k = 0; k < 3; ++k) o->axis[k] = axis[k] / n;
    o->alpha = alpha;
    o->gamma = gamma;
}

/* Applied field: uniform part hu * s(t) and optional cell part hcell * s_c(t), with
 * s(t) = 1 for freq == 0 and sin(2 pi freq t + phase) otherwise. */
void or_set_zeeman(void *h, const double *hu, double hu_freq, double hu_phase, const double *hcell,
                   double hc_freq, double hc_phase)
{
    OrMesh *o = (OrMesh *)h;
    for (int k = 0; k < 3; ++k) o->hu[k] = hu[k];
    o->hu_freq = hu_freq; o->hu_phase = hu_phase;
    free(o->hcell);
    o->hcell = NULL;
    if (hcell) {
        long nc = n_cells(o);
        o->hcell = (double *)malloc(nc * 3 * sizeof(double));
        memcpy(o->hcell, hcell, nc * 3 * sizeof(double));
    }
    o->hc_freq = hc_freq; o->hc_phase = hc_phase;
}

static double time_factor(double freq, double phase, double t)
{
    return freq == 0.0 ? 1.0 : sin(2.0 * M_PI * freq * t + phase);
}

/* ------------------------------------------------------------------------------------------------
 * Lumped mass (Eq. mass_lumping): mass_n = int mu0 Ms^h phi_n dx = sum_{c ∋ n} mu0 Ms_c int_c phi
 * ---------------------------------------------------------------------------------------------- */
void or_mass(void *h, double *mass)
{
    OrMesh *o = (OrMesh *)h;
    long nn = n_nodes(o);
    for (long n = 0; n < nn; ++n) mass[n] = 0.0;
    for (int c1 = 0; c1 < o->N[0]; ++c1)
        for (int c2 = 0; c2 < o->N[1]; ++c2)
            for (int c3 = 0; c3 < o->N[2]; ++c3) {
                double Ms = o->Ms[cidx(o, c1, c2, c3)];
                for (int li = 0; li < 8; ++li) {
                    int i[3];
                    vertex_of(li, i);
                    mass[nidx(o, c1 + i[0], c2 + i[1], c3 + i[2])] += MU0 * Ms * o->Phi[li];
                }
            }
}

/* ------------------------------------------------------------------------------------------------
 * Newell tensor (Newell, Williams & Dunlop 1993) of two identical cuboids dx1 x dx2 x dx3 at offset
 * (X, Y, Z), in _Float128.  f and g are the published auxiliary functions; the tensor is the
 * 27-point second difference (weights -1, 2, -1 per direction) divided by 4 pi V.
 * ---------------------------------------------------------------------------------------------- */
static q128 newell_f(q128 x, q128 y, q128 z)
{
    q128 x2 = x * x, y2 = y * y, z2 = z * z;
    q128 R = sqrtf128(x2 + y2 + z2);
    q128 r = 0;
    if (x2 + z2 > 0) r += y / 2 * (z2 - x2) * asinhf128(y / sqrtf128(x2 + z2));
    if (x2 + y2 > 0) r += z / 2 * (y2 - x2) * asinhf128(z / sqrtf128(x2 + y2));
    if (x != 0 && y != 0 && z != 0) r -= x * y * z * atanf128(y * z / (x * R));
    r += (2 * x2 - y2 - z2) * R / 6;
    return r;
}

static q128 newell_g(q128 x, q128 y, q128 z)
{
    q128 x2 = x * x, y2 = y * y, z2 = z * z;
    q128 R = sqrtf128(x2 + y2 + z2);
    q128 r = 0;
    if (x != 0 && y != 0) r += x * y * z * asinhf128(z / sqrtf128(x2 + y2));
    if (y2 + z2 > 0) r += y / 6 * (3 * z2 - y2) * asinhf128(x / sqrtf128(y2 + z2));
    if (x2 + z2 > 0) r += x / 6 * (3 * z2 - x2) * asinhf128(y / sqrtf128(x2 + z2));
    if (z != 0 && x != 0 && y != 0) r -= z * z2 / 6 * atanf128(x * y / (z * R));
    if (y != 0 && x != 0 && z != 0) r -= z * y2 / 2 * atanf128(x * z / (y * R));
    if (x != 0 && y != 0 && z != 0) r -= z * x2 / 2 * atanf128(y * z / (x * R));
    r -= x * y * R / 3;
    return r;
}

/* out = (Nxx, Nyy, Nzz, Nxy, Nxz, Nyz) */
void or_newell(double dx1, double dx2, double dx3, double X, double Y, double Z, double *out)
{
    const q128 d[3] = {dx1, dx2, dx3};
    const q128 P[3] = {X, Y, Z};
    q128 s[6] = {0, 0, 0, 0, 0, 0};
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
            for (int c = -1; c <= 1; ++c) {
                q128 w = (q128)((a == 0 ? 2 : -1) * (b == 0 ? 2 : -1) * (c == 0 ? 2 : -1));
                q128 x = P[0] + a * d[0], y = P[1] + b * d[1], z = P[2] + c * d[2];
                s[0] += w * newell_f(x, y, z);
                s[1] += w * newell_f(y, z, x);
                s[2] += w * newell_f(z, x, y);
                s[3] += w * newell_g(x, y, z);
                s[4] += w * newell_g(x, z, y);
                s[5] += w * newell_g(y, z, x);
            }
    const q128 pi_q = 3.14159265358979323846264338327950288f128;
    q128 den = 4 * pi_q * d[0] * d[1] * d[2];
    for (int k = 0; k < 6; ++k) out[k] = (double)(s[k] / den);
}

/* Octant of the tensor for all cell offsets (d1, d2, d3) in [0,N1) x [0,N2) x [0,N3). */
void or_compute_tensor(void *h)
{
    OrMesh *o = (OrMesh *)h;
    long nc = n_cells(o);
    if (!o->Nt) o->Nt = (double *)malloc(nc * 6 * sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
    for (long c = 0; c < nc; ++c) {
        int d3 = (int)(c % o->N[2]);
        int d2 = (int)((c / o->N[2]) % o->N[1]);
        int d1 = (int)(c / ((long)o->N[2] * o->N[1]));
        or_newell(o->dx[0], o->dx[1], o->dx[2], d1 * o->dx[0], d2 * o->dx[1], d3 * o->dx[2], o->Nt + 6 * c);
    }
}

void or_get_tensor(void *h, double *out)
{
    OrMesh *o = (OrMesh *)h;
    if (!o->Nt) or_compute_tensor(h);
    memcpy(out, o->Nt, n_cells(o) * 6 * sizeof(double));
}

/* N at signed offset (e1,e2,e3): diagonal entries are even in each offset; Nxy is odd in e1 and e2,
 * Nxz odd in e1 and e3, Nyz odd in e2 and e3. */
static void tensor_at(const OrMesh *o, int e1, int e2, int e3, double N[6])
{
    const double *t = o->Nt + 6 * cidx(o, abs(e1), abs(e2), abs(e3));
    int s1 = e1 < 0 ? -1 : 1, s2 = e2 < 0 ? -1 : 1, s3 = e3 < 0 ? -1 : 1;
    N[0] = t[0]; N[1] = t[1]; N[2] = t[2];
    N[3] = s1 * s2 * t[3];
    N[4] = s1 * s3 * t[4];
    N[5] = s2 * s3 * t[5];
}

/* Cell mean of the nodal interpolant, m_bar_c = (1/V) int_c m^h (the node->cell averaging of the
 * demag pre-processing step), by Gauss quadrature of the interpolant. */
static void cell_mean(const OrMesh *o, const double *m, int c1, int c2, int c3, double mb[3])
{
    mb[0] = mb[1] = mb[2] = 0.0;
    for (int q = 0; q < 8; ++q) {
        double xi[3], w;
        gauss_point(q, xi, &w);
        for (int li = 0; li < 8; ++li) {
            int i[3];
            vertex_of(li, i);
            double p = or_phi(li, xi[0], xi[1], xi[2]);
            const double *mv = m + 3 * nidx(o, c1 + i[0], c2 + i[1], c3 + i[2]);
            for (int j = 0; j < 3; ++j) mb[j] += w * p * mv[j];
        }
    }
}

/* Cell demag field H_c = - sum_{c'} N(c - c') Ms_c' m_bar_c'  (direct sum; cells x 3). */
void or_demag_cells(void *h, const double *m, double *Hc)
{
    OrMesh *o = (OrMesh *)h;
    if (!o->Nt) or_compute_tensor(h);
    long nc = n_cells(o);
    double *M = (double *)malloc(nc * 3 * sizeof(double));
    for (int c1 = 0; c1 < o->N[0]; ++c1)
        for (int c2 = 0; c2 < o->N[1]; ++c2)
            for (int c3 = 0; c3 < o->N[2]; ++c3) {
                long c = cidx(o, c1, c2, c3);
                double mb[3];
                cell_mean(o, m, c1, c2, c3, mb);
                for (int j = 0; j < 3; ++j) M[3 * c + j] = o->Ms[c] * mb[j];
            }
#pragma omp parallel for schedule(dynamic, 16)
    for (long c = 0; c < nc; ++c) {
        int c3 = (int)(c % o->N[2]);
        int c2 = (int)((c / o->N[2]) % o->N[1]);
        int c1 = (int)(c / ((long)o->N[2] * o->N[1]));
        double H[3] = {0.0, 0.0, 0.0};
        for (int b1 = 0; b1 < o->N[0]; ++b1)
            for (int b2 = 0; b2 < o->N[1]; ++b2)
                for (int b3 = 0; b3 < o->N[2]; ++b3) {
                    const double *Mb = M + 3 * cidx(o, b1, b2, b3);
                    double N[6];
                    tensor_at(o, c1 - b1, c2 - b2, c3 - b3, N);
                    H[0] -= N[0] * Mb[0] + N[3] * Mb[1] + N[4] * Mb[2];
                    H[1] -= N[3] * Mb[0] + N[1] * Mb[1] + N[5] * Mb[2];
                    H[2] -= N[4] * Mb[0] + N[5] * Mb[1] + N[2] * Mb[2];
                }
        for (int j = 0; j < 3; ++j) Hc[3 * c + j] = H[j];
    }
    free(M);
}

/* ------------------------------------------------------------------------------------------------
 * Variation dE_{n,j} = dE(m^h, phi_{n,j}) assembled cell by cell (Eqs. weak_form_impl_f and
 * weak_form_impl: the cell c contributes to node n = c + i through its element integrals).
 *   exchange    E = int A |grad m|^2            ->  A_c  sum_i' Kex(i,i') m_{c+i'}
 *   anisotropy  E = -int Ku (m.e)^2             -> -2 Ku_c e sum_i' Mm(i,i') (e . m_{c+i'})
 *   Zeeman      E = -mu0 int Ms h.m             -> -mu0 Ms_c h_c int_c phi_i
 *   demag       dE(m,v) = -mu0 int Ms H_d . v   -> -mu0 Ms_c H_c int_c phi_i
 * ---------------------------------------------------------------------------------------------- */
void or_variation(void *h, const double *m, unsigned terms, double t, double *dE)
{
    OrMesh *o = (OrMesh *)h;
    long nn = n_nodes(o), nc = n_cells(o);
    for (long a = 0; a < 3 * nn; ++a) dE[a] = 0.0;
    double *Hc = NULL;
    if (terms & TERM_DEMAG) {
        Hc = (double *)malloc(nc * 3 * sizeof(double));
        or_demag_cells(h, m, Hc);
    }
    const double su = time_factor(o->hu_freq, o->hu_phase, t);
    const double sc = time_factor(o->hc_freq, o->hc_phase, t);
    const double *e = o->axis;
    for (int c1 = 0; c1 < o->N[0]; ++c1)
        for (int c2 = 0; c2 < o->N[1]; ++c2)
            for (int c3 = 0; c3 < o->N[2]; ++c3) {
                long c = cidx(o, c1, c2, c3);
                if (o->Ms[c] == 0.0) continue; /* vacuum */
                const double *mc[8];
                for (int lj = 0; lj < 8; ++lj) {
                    int i[3];
                    vertex_of(lj, i);
                    mc[lj] = m + 3 * nidx(o, c1 + i[0], c2 + i[1], c3 + i[2]);
                }
                for (int li = 0; li < 8; ++li) {
                    int i[3];
                    vertex_of(li, i);
                    double *d = dE + 3 * nidx(o, c1 + i[0], c2 + i[1], c3 + i[2]);
                    if (terms & TERM_EXCH)
                        for (int lj = 0; lj < 8; ++lj)
                            for (int j = 0; j < 3; ++j) d[j] += o->A[c] * o->Kex[li][lj] * mc[lj][j];
                    if (terms & TERM_ANIS)
                        for (int lj = 0; lj < 8; ++lj) {
                            double em = e[0] * mc[lj][0] + e[1] * mc[lj][1] + e[2] * mc[lj][2];
                            for (int j = 0; j < 3; ++j) d[j] += -2.0 * o->Ku[c] * e[j] * o->Mm[li][lj] * em;
                        }
                    if (terms & TERM_ZEE)
                        for (int j = 0; j < 3; ++j) {
                            double hj = o->hu[j] * su + (o->hcell ? o->hcell[3 * c + j] * sc : 0.0);
                            d[j] += -MU0 * o->Ms[c] * hj * o->Phi[li];
                        }
                    if (terms & TERM_DEMAG)
                        for (int j = 0; j < 3; ++j) d[j] += -MU0 * o->Ms[c] * Hc[3 * c + j] * o->Phi[li];
                    if ((terms & TERM_DMI) && o->D[c] != 0.0)
                        /* E_c = D sum_{i,i'} [m_iz G_x(i,i') m_i'x + m_iz G_y(i,i') m_i'y
                         *                     - m_ix G_x(i,i') m_i'z - m_iy G_y(i,i') m_i'z] */
                        for (int lj = 0; lj < 8; ++lj) {
                            const double ax = o->Gd[0][li][lj] - o->Gd[0][lj][li];
                            const double ay = o->Gd[1][li][lj] - o->Gd[1][lj][li];
                            d[0] += -o->D[c] * ax * mc[lj][2];
                            d[1] += -o->D[c] * ay * mc[lj][2];
                            d[2] += o->D[c] * (ax * mc[lj][0] + ay * mc[lj][1]);
                        }
                }
            }
    free(Hc);
}

/* Effective field with mass lumping (Eq. mass_lumping): H_{n,j} = -dE_{n,j} / mass_n, and 0 on
 * nodes that touch no magnetic cell. */
void or_h_eff(void *h, const double *m, unsigned terms, double t, double *H)
{
    OrMesh *o = (OrMesh *)h;
    long nn = n_nodes(o);
    double *mass = (double *)malloc(nn * sizeof(double));
    or_mass(h, mass);
    or_variation(h, m, terms, t, H);
    for (long n = 0; n < nn; ++n)
        for (int j = 0; j < 3; ++j) H[3 * n + j] = mass[n] > 0.0 ? -H[3 * n + j] / mass[n] : 0.0;
    free(mass);
}

/* Energies, evaluated from their definitions by Gauss quadrature of the nodal interpolant
 * (independent of the element matrices above): Eq. exchange_energy, anisotropy -int Ku (m.e)^2,
 * Zeeman -mu0 int Ms h.m, demag -(mu0/2) int Ms m.H_d with cell-constant H_d. */
double or_energy(void *h, const double *m, unsigned terms, double t)
{
    OrMesh *o = (OrMesh *)h;
    long nc = n_cells(o);
    double *Hc = NULL;
    if (terms & TERM_DEMAG) {
        Hc = (double *)malloc(nc * 3 * sizeof(double));
        or_demag_cells(h, m, Hc);
    }
    const double V = o->dx[0] * o->dx[1] * o->dx[2];
    const double su = time_factor(o->hu_freq, o->hu_phase, t);
    const double sc = time_factor(o->hc_freq, o->hc_phase, t);
    double E = 0.0;
    for (int c1 = 0; c1 < o->N[0]; ++c1)
        for (int c2 = 0; c2 < o->N[1]; ++c2)
            for (int c3 = 0; c3 < o->N[2]; ++c3) {
                long c = cidx(o, c1, c2, c3);
                if (o->Ms[c] == 0.0) continue;
                for (int q = 0; q < 8; ++q) {
                    double xi[3], w;
                    gauss_point(q, xi, &w);
                    double mv[3] = {0, 0, 0}, gm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                    for (int li = 0; li < 8; ++li) {
                        int i[3];
                        vertex_of(li, i);
                        const double *mn = m + 3 * nidx(o, c1 + i[0], c2 + i[1], c3 + i[2]);
                        double p = or_phi(li, xi[0], xi[1], xi[2]);
                        double g[3];
                        grad_phi(li, xi, o->dx, g);
                        for (int j = 0; j < 3; ++j) {
                            mv[j] += p * mn[j];
                            for (int k = 0; k < 3; ++k) gm[j][k] += mn[j] * g[k];
                        }
                    }
                    double dV = w * V;
                    if (terms & TERM_EXCH) {
                        double s = 0.0;
                        for (int j = 0; j < 3; ++j)
                            for (int k = 0; k < 3; ++k) s += gm[j][k] * gm[j][k];
                        E += o->A[c] * s * dV;
                    }
                    if (terms & TERM_ANIS) {
                        double em = o->axis[0] * mv[0] + o->axis[1] * mv[1] + o->axis[2] * mv[2];
                        E += -o->Ku[c] * em * em * dV;
                    }
                    if (terms & TERM_ZEE)
                        for (int j = 0; j < 3; ++j) {
                            double hj = o->hu[j] * su + (o->hcell ? o->hcell[3 * c + j] * sc : 0.0);
                            E += -MU0 * o->Ms[c] * hj * mv[j] * dV;
                        }
                    if (terms & TERM_DEMAG)
                        for (int j = 0; j < 3; ++j) E += -0.5 * MU0 * o->Ms[c] * Hc[3 * c + j] * mv[j] * dV;
                    if (terms & TERM_DMI)  /* gm[j][k] = d_k m_j */
                        E += o->D[c] * (mv[2] * (gm[0][0] + gm[1][1]) - mv[0] * gm[2][0] - mv[1] * gm[2][1]) * dV;
                }
            }
    free(Hc);
    return E;
}

/* ------------------------------------------------------------------------------------------------
 * LLG right-hand side (Eq. llg):
 *   dm/dt = -gamma/(1+alpha^2) m x H - alpha gamma/(1+alpha^2) m x (m x H),
 * zero on nodes without magnetic material.
 * ---------------------------------------------------------------------------------------------- */
static void cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

void or_llg_rhs(void *h, const double *m, unsigned terms, double t, double *k)
{
    OrMesh *o = (OrMesh *)h;
    long nn = n_nodes(o);
    double *H = (double *)malloc(nn * 3 * sizeof(double));
    double *mass = (double *)malloc(nn * sizeof(double));
    or_h_eff(h, m, terms, t, H);
    or_mass(h, mass);
    const double g = o->gamma / (1.0 + o->alpha * o->alpha);
    for (long n = 0; n < nn; ++n) {
        double mxH[3], mxmxH[3];
        cross(m + 3 * n, H + 3 * n, mxH);
        cross(m + 3 * n, mxH, mxmxH);
        for (int j = 0; j < 3; ++j)
            k[3 * n + j] = mass[n] > 0.0 ? -g * mxH[j] - o->alpha * g * mxmxH[j] : 0.0;
    }
    free(H);
    free(mass);
}

static void renormalise(const OrMesh *o, double *m)
{
    long nn = n_nodes(o);
    for (long n = 0; n < nn; ++n) {
        double s = sqrt(m[3 * n] * m[3 * n] + m[3 * n + 1] * m[3 * n + 1] + m[3 * n + 2] * m[3 * n + 2]);
        if (s > 0.0)
            for (int j = 0; j < 3; ++j) m[3 * n + j] /= s;
    }
}

/* Classical fourth-order Runge-Kutta step; optional renormalisation of |m| afterwards. */
void or_rk4_step(void *h, double *m, unsigned terms, double t, double dt, int renorm)
{
    OrMesh *o = (OrMesh *)h;
    long n3 = 3 * n_nodes(o);
    double *k1 = malloc(n3 * sizeof(double)), *k2 = malloc(n3 * sizeof(double));
    double *k3 = malloc(n3 * sizeof(double)), *k4 = malloc(n3 * sizeof(double));
    double *y = malloc(n3 * sizeof(double));
    or_llg_rhs(h, m, terms, t, k1);
    for (long a = 0; a < n3; ++a) y[a] = m[a] + 0.5 * dt * k1[a];
    or_llg_rhs(h, y, terms, t + 0.5 * dt, k2);
    for (long a = 0; a < n3; ++a) y[a] = m[a] + 0.5 * dt * k2[a];
    or_llg_rhs(h, y, terms, t + 0.5 * dt, k3);
    for (long a = 0; a < n3; ++a) y[a] = m[a] + dt * k3[a];
    or_llg_rhs(h, y, terms, t + dt, k4);
    for (long a = 0; a < n3; ++a) m[a] += dt / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
    if (renorm) renormalise(o, m);
    free(k1); free(k2); free(k3); free(k4); free(y);
}

/* Dormand & Prince (1980) RK5(4)7M tableau. */
static const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
/* fifth-order weights (= last row of A) and fourth-order embedded weights */
static const double DP_B[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
static const double DP_BS[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200,
                                187.0 / 2100, 1.0 / 40};

void or_dp5_tableau(double *c, double *a, double *b, double *bs)
{
    for (int i = 0; i < 7; ++i) {
        c[i] = DP_C[i];
        b[i] = DP_B[i];
        bs[i] = DP_BS[i];
        for (int j = 0; j < 6; ++j) a[i * 6 + j] = DP_A[i][j];
    }
}

/* One adaptive Dormand-Prince step with FSAL.
 *  k1      in: f(t, m) (computed when *k1_valid == 0); out: f at the new point when accepted.
 *  error   err = RMS over magnetic nodes and components of (dt sum_i e_i k_i) / (atol + rtol max(|m|,|m5|))
 *  control accept when err <= 1; dt <- dt * clamp(0.9 err^(-1/5), 0.2, 5); a non-finite err rejects
 *          with factor 0.2.
 *  accept  t += dt, m <- m5 (renormalised when renorm != 0), k1 <- k7 (FSAL, taken at m5 before
 *          renormalisation).
 * Returns 1 when accepted. */
int or_dp5_step(void *h, double *m, double *k1, int *k1_valid, unsigned terms, double *t, double *dt,
                double rtol, double atol, int renorm, double *err_out)
{
    OrMesh *o = (OrMesh *)h;
    long nn = n_nodes(o), n3 = 3 * nn;
    double *k[7];
    k[0] = k1;
    for (int s = 1; s < 7; ++s) k[s] = malloc(n3 * sizeof(double));
    double *y = malloc(n3 * sizeof(double));
    double *mass = malloc(nn * sizeof(double));
    or_mass(h, mass);
    const double h_ = *dt, t0 = *t;
    if (!*k1_valid) {
        or_llg_rhs(h, m, terms, t0, k1);
        *k1_valid = 1;
    }
    for (int s = 1; s < 7; ++s) {
        for (long a = 0; a < n3; ++a) {
            double acc = 0.0;
            for (int j = 0; j < s; ++j) acc += DP_A[s][j] * k[j][a];
            y[a] = m[a] + h_ * acc;
        }
        or_llg_rhs(h, y, terms, t0 + DP_C[s] * h_, k[s]);
    }
    /* y now holds m5 = m + dt sum b_j k_j (stage 7 input) */
    double sum = 0.0;
    long cnt = 0;
    for (long n = 0; n < nn; ++n) {
        if (!(mass[n] > 0.0)) continue;
        for (int j = 0; j < 3; ++j) {
            long a = 3 * n + j;
            double ev = 0.0;
            for (int s = 0; s < 7; ++s) ev += (DP_B[s] - DP_BS[s]) * k[s][a];
            ev *= h_;
            double sc = atol + rtol * fmax(fabs(m[a]), fabs(y[a]));
            sum += (ev / sc) * (ev / sc);
            ++cnt;
        }
    }
    double err = cnt ? sqrt(sum / cnt) : 0.0;
    if (err_out) *err_out = err;
    int acc = isfinite(err) && err <= 1.0;
    double fac;
    if (!isfinite(err)) fac = 0.2;
    else if (err == 0.0) fac = 5.0;
    else fac = fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2)));
    if (acc) {
        memcpy(m, y, n3 * sizeof(double));
        if (renorm) renormalise(o, m);
        memcpy(k1, k[6], n3 * sizeof(double));
        *t = t0 + h_;
    }
    *dt = h_ * fac;
    for (int s = 1; s < 7; ++s) free(k[s]);
    free(y);
    free(mass);
    return acc;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of the parallel loops that follow (for timing: each iteration of those loops writes its
   own outputs from sums taken in a fixed order, so the results do not depend on it). */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
