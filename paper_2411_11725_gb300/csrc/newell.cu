// Demag tensor set-up (FP64, once per mesh): the cell-averaged field tensor of two homogeneously
// magnetised cuboids (the standard finite-difference demag kernel the paper's "Demagnetization Field"
// section builds on), and its spectrum on the padded grid.
//
// Near offsets use the closed form of Newell, Williams & Dunlop (1993).  Its 27-term second
// difference cancels catastrophically with distance (relative error ~ eps (r/dx)^6 in FP64), so
// farther offsets integrate the point-dipole kernel against the triangle density of the difference
// of two points of the cells, -(V/4 pi) E[(3 r r^T / r^2 - I) / r^3], with a tensor-product
// Gauss-Legendre rule on each half of the triangle; the integrand is analytic there and the rule
// converges geometrically.
//
// The spectrum is computed one direction at a time: each component is even or odd along each
// direction, so its transform along that direction is a cosine or sine transform of the octant data,
// evaluated as a complex FFT of the symmetrically extended line (real part for even, imaginary part
// for odd), keeping the non-negative half of the frequencies.
#include <math.h>

#include <vector>

#include "fft.cuh"
#include "newell.cuh"

namespace nm {

// ------------------------------------------------------------------------------ Newell closed form
__device__ double nw_f(double x, double y, double z)
{
    const double xx = x * x, yy = y * y, zz = z * z;
    const double R = sqrt(xx + yy + zz);
    double r = (2.0 * xx - yy - zz) * R / 6.0;
    if (xx + zz > 0.0) r += 0.5 * y * (zz - xx) * asinh(y / sqrt(xx + zz));
    if (xx + yy > 0.0) r += 0.5 * z * (yy - xx) * asinh(z / sqrt(xx + yy));
    if (x != 0.0 && y != 0.0 && z != 0.0) r -= x * y * z * atan(y * z / (x * R));
    return r;
}

__device__ double nw_g(double x, double y, double z)
{
    const double xx = x * x, yy = y * y, zz = z * z;
    const double R = sqrt(xx + yy + zz);
    double r = -x * y * R / 3.0;
    if (x != 0.0 && y != 0.0) r += x * y * z * asinh(z / sqrt(xx + yy));
    if (yy + zz > 0.0) r += y / 6.0 * (3.0 * zz - yy) * asinh(x / sqrt(yy + zz));
    if (xx + zz > 0.0) r += x / 6.0 * (3.0 * zz - xx) * asinh(y / sqrt(xx + zz));
    if (x != 0.0 && y != 0.0 && z != 0.0) {
        r -= zz * z / 6.0 * atan(x * y / (z * R));
        r -= 0.5 * z * yy * atan(x * z / (y * R));
        r -= 0.5 * z * xx * atan(y * z / (x * R));
    }
    return r;
}

__device__ void newell_closed(double X, double Y, double Z, double a, double b, double c, double out[6])
{
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int p = -1; p <= 1; ++p) {
        const double wx = p == 0 ? 2.0 : -1.0, x = X + p * a;
        for (int q = -1; q <= 1; ++q) {
            const double wy = q == 0 ? 2.0 : -1.0, y = Y + q * b;
            for (int r = -1; r <= 1; ++r) {
                const double w = wx * wy * (r == 0 ? 2.0 : -1.0), z = Z + r * c;
                s[0] += w * nw_f(x, y, z);
                s[1] += w * nw_f(y, z, x);
                s[2] += w * nw_f(z, x, y);
                s[3] += w * nw_g(x, y, z);
                s[4] += w * nw_g(x, z, y);
                s[5] += w * nw_g(y, z, x);
            }
        }
    }
    const double den = 4.0 * 3.14159265358979323846 * a * b * c;
    for (int k = 0; k < 6; ++k) out[k] = s[k] / den;
}

// ------------------------------------------------------------------------------ far-field quadrature
struct TentRule {
    double s[4][32];  // symmetric nodes on [-1, 1] for the rules of 4, 6, 10, 16 points per half
    double w[4][32];  // weights: sum w = 1 for each rule, density (1 - |s|)
    int n[4];
};

__device__ void newell_quad(double X, double Y, double Z, double a, double b, double c, const TentRule &tr, int ri,
                            double out[6])
{
    double s[6] = {0, 0, 0, 0, 0, 0};
    const int n = tr.n[ri];
    for (int i = 0; i < n; ++i) {
        const double x = X + tr.s[ri][i] * a, wi = tr.w[ri][i];
        for (int j = 0; j < n; ++j) {
            const double y = Y + tr.s[ri][j] * b, wij = wi * tr.w[ri][j];
            for (int k = 0; k < n; ++k) {
                const double z = Z + tr.s[ri][k] * c, w = wij * tr.w[ri][k];
                const double r2 = x * x + y * y + z * z;
                const double ir2 = 1.0 / r2;
                const double ir3 = ir2 / sqrt(r2);
                const double q = w * ir3;
                const double q3 = 3.0 * q * ir2;
                s[0] += q3 * x * x - q;
                s[1] += q3 * y * y - q;
                s[2] += q3 * z * z - q;
                s[3] += q3 * x * y;
                s[4] += q3 * x * z;
                s[5] += q3 * y * z;
            }
        }
    }
    const double f = -a * b * c / (4.0 * 3.14159265358979323846);
    for (int k = 0; k < 6; ++k) out[k] = f * s[k];
}

// One thread per offset (d1, d2, d3) of the octant; output W[comp][d3][d2][d1].
__global__ void k_newell_octant(int N1, int N2, int N3, double a, double b, double c, TentRule tr, double *W)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long nc = (long)N1 * N2 * N3;
    if (i >= nc) return;
    const int d1 = (int)(i % N1);
    const int d2 = (int)((i / N1) % N2);
    const int d3 = (int)(i / ((long)N1 * N2));
    const double X = d1 * a, Y = d2 * b, Z = d3 * c;
    const double hmax = fmax(a, fmax(b, c));
    const double rho = sqrt(X * X + Y * Y + Z * Z) / hmax;
    double out[6];
    if (rho < 2.5) newell_closed(X, Y, Z, a, b, c, out);
    else newell_quad(X, Y, Z, a, b, c, tr, rho < 5.0 ? 3 : (rho < 10.0 ? 2 : (rho < 32.0 ? 1 : 0)), out);
    for (int k = 0; k < 6; ++k) W[k * nc + i] = out[k];
}

// Symmetric line transform: line l = (comp, u, v), in[j] for j < N at in_base + j*in_es; output
// k < H = P/2+1 at out_base + k*out_es.  Even components take Re, odd ones Im of the FFT of the
// extended line g[j] = f(j), g[P-j] = +-f(j).
struct LineMap {
    long in_cs, in_as, in_bs, in_es;
    long out_cs, out_as, out_bs, out_es;
    int na, nb;
    int N, P, lgP, H;
    int parity[6];  // +1 even, -1 odd, per component
};

__global__ void __launch_bounds__(512, 1) k_sym_lines(LineMap lm, const double *__restrict__ in, double *__restrict__ out,
                                                   const Cx<double> *__restrict__ tw, int twlg, int lpb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<double> *buf = reinterpret_cast<Cx<double> *>(smem_raw);
    const long nlines = 6L * lm.na * lm.nb;
    const long l0 = (long)blockIdx.x * lpb;
    const int nl = (int)min((long)lpb, nlines - l0);
    if (nl <= 0) return;
    const int P = lm.P, lsz = padded_len(P);
    auto line = [&](int li, int &comp, long &ib, long &ob) {
        long l = l0 + li;
        comp = (int)(l / ((long)lm.na * lm.nb));
        long rem = l % ((long)lm.na * lm.nb);
        int ua = (int)(rem / lm.nb), vb = (int)(rem % lm.nb);
        ib = comp * lm.in_cs + ua * lm.in_as + vb * lm.in_bs;
        ob = comp * lm.out_cs + ua * lm.out_as + vb * lm.out_bs;
    };
    // extended line g[j] = f(j) for j < N, g[P - j] = parity * f(j) for 0 < j < N, else 0
    auto src = [&](int li, int j) -> Cx<double> {
        int comp;
        long ib, ob;
        line(li, comp, ib, ob);
        double v = 0.0;
        if (j < lm.N) v = in[ib + j * lm.in_es];
        else if (P - j < lm.N) v = lm.parity[comp] * in[ib + (P - j) * lm.in_es];
        return cx<double>(v, 0.0);
    };
    auto sm = [&](int li, int i) { return li * lsz + pad16(i); };
    auto dst = [&](int li, int k, Cx<double> z) {
        int comp;
        long ib, ob;
        line(li, comp, ib, ob);
        out[ob + k * lm.out_es] = lm.parity[comp] > 0 ? z.x : z.y;
    };
    fft_lines<double, false, false, false>(buf, FastDiv((unsigned)nl), lm.lgP, -1, tw, twlg, P, lm.H, src, sm, dst);
}

template <typename T>
__global__ void k_tensor_final(long n, long comp_stride, const double *__restrict__ W, double scale, T *__restrict__ Nk)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= 6 * n) return;
    int comp = (int)(i / n);
    long j = i % n;
    // H = -N * M: diagonal components -1, off-diagonal ones carry (-i)^2 = -1 from the two sine
    // transforms, so their sign flips back.
    double s = comp < 3 ? -scale : scale;
    Nk[comp * comp_stride + j] = (T)(s * W[comp * n + j]);
}

// ------------------------------------------------------------------------------ host
// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n (long double).
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        long double z = cosl(pi * (i + 0.75L) / (n + 0.5L)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1);
            long double dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < 1e-30L) break;
        }
        x[i] = (double)z;
        w[i] = (double)(2.0L / ((1 - z * z) * dp * dp));
    }
}

static TentRule make_tent_rule()
{
    TentRule tr;
    const int q[4] = {4, 6, 10, 16};
    for (int r = 0; r < 4; ++r) {
        std::vector<double> x, w;
        gauss_legendre(q[r], x, w);
        int n = 0;
        for (int i = 0; i < q[r]; ++i) {
            // node on [0, 1]: u = (x + 1)/2, weight w/2; density (1 - u) on each half
            double u = 0.5 * (x[i] + 1.0), wu = 0.5 * w[i] * (1.0 - u);
            tr.s[r][n] = u;
            tr.w[r][n++] = wu;
            tr.s[r][n] = -u;
            tr.w[r][n++] = wu;
        }
        tr.n[r] = n;
    }
    return tr;
}

static int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

static cudaError_t sym_pass(const LineMap &lm, const double *in, double *out, const Cx<double> *tw, int twlg,
                            cudaStream_t st)
{
    // lines per block within the FFT engine's budget: lpb * P <= fft_regs<double>() * threads
    int lpb = fft_regs<double>() * 512 / lm.P;
    if (lpb < 1) return cudaErrorInvalidConfiguration;
    if (lpb > 64) lpb = 64;
    size_t sm = (size_t)lpb * padded_len(lm.P) * sizeof(Cx<double>);
    cudaFuncSetAttribute(k_sym_lines, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    long nlines = 6L * lm.na * lm.nb;
    const int nt = 512;
    k_sym_lines<<<(int)((nlines + lpb - 1) / lpb), nt, sm, st>>>(lm, in, out, tw, twlg, lpb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t build_tensor_spectrum(const Geom &g, double a, double b, double c, const Cx<double> *tw64, T *Nk,
                                  cudaStream_t st)
{
    const long nc = (long)g.N1 * g.N2 * g.N3;
    const long sz1 = 6 * nc;
    const long sz2 = 6L * g.N3 * g.N2 * g.Xp;
    const long sz3 = 6L * g.N3 * g.H2 * g.Xp;
    const long sz4 = 6L * g.H3 * g.H2 * g.Xp;
    long szA = sz1 > sz3 ? sz1 : sz3;
    long szB = sz2 > sz4 ? sz2 : sz4;
    double *A = nullptr, *B = nullptr;
    cudaError_t e = cudaMallocAsync(&A, szA * sizeof(double), st);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync(&B, szB * sizeof(double), st);
    if (e != cudaSuccess) { cudaFreeAsync(A, st); return e; }
    cudaMemsetAsync(B, 0, szB * sizeof(double), st);
    TentRule tr = make_tent_rule();
    k_newell_octant<<<div_up(nc, 128), 128, 0, st>>>(g.N1, g.N2, g.N3, a, b, c, tr, A);
    const int par[3][6] = {{1, 1, 1, -1, -1, 1}, {1, 1, 1, -1, 1, -1}, {1, 1, 1, 1, -1, -1}};
    // x: A [6][N3][N2][N1] -> B [6][N3][N2][Xp]
    LineMap lm{};
    lm.na = g.N3; lm.nb = g.N2;
    lm.in_cs = nc; lm.in_as = (long)g.N2 * g.N1; lm.in_bs = g.N1; lm.in_es = 1;
    lm.out_cs = (long)g.N3 * g.N2 * g.Xp; lm.out_as = (long)g.N2 * g.Xp; lm.out_bs = g.Xp; lm.out_es = 1;
    lm.N = g.N1; lm.P = g.P1; lm.lgP = ilog2(g.P1); lm.H = g.P1 / 2 + 1;
    for (int k = 0; k < 6; ++k) lm.parity[k] = par[0][k];
    if ((e = sym_pass(lm, A, B, tw64, g.twlg, st)) != cudaSuccess) goto done;
    // y: B [6][N3][N2][Xp] -> A [6][N3][H2][Xp]
    lm.na = g.N3; lm.nb = g.Xp;
    lm.in_cs = (long)g.N3 * g.N2 * g.Xp; lm.in_as = (long)g.N2 * g.Xp; lm.in_bs = 1; lm.in_es = g.Xp;
    lm.out_cs = (long)g.N3 * g.H2 * g.Xp; lm.out_as = (long)g.H2 * g.Xp; lm.out_bs = 1; lm.out_es = g.Xp;
    lm.N = g.N2; lm.P = g.P2; lm.lgP = ilog2(g.P2); lm.H = g.H2;
    for (int k = 0; k < 6; ++k) lm.parity[k] = par[1][k];
    if ((e = sym_pass(lm, B, A, tw64, g.twlg, st)) != cudaSuccess) goto done;
    // z: A [6][N3][H2][Xp] -> B [6][H3][H2][Xp]
    lm.na = g.H2; lm.nb = g.Xp;
    lm.in_cs = (long)g.N3 * g.H2 * g.Xp; lm.in_as = g.Xp; lm.in_bs = 1; lm.in_es = (long)g.H2 * g.Xp;
    lm.out_cs = (long)g.H3 * g.H2 * g.Xp; lm.out_as = g.Xp; lm.out_bs = 1; lm.out_es = (long)g.H2 * g.Xp;
    lm.N = g.N3; lm.P = g.P3; lm.lgP = ilog2(g.P3); lm.H = g.H3;
    for (int k = 0; k < 6; ++k) lm.parity[k] = par[2][k];
    if ((e = sym_pass(lm, A, B, tw64, g.twlg, st)) != cudaSuccess) goto done;
    {
        long n = (long)g.H3 * g.H2 * g.Xp;
        double scale = 1.0 / ((double)g.P1 * g.P2 * g.P3);
        k_tensor_final<T><<<div_up(6 * n, 256), 256, 0, st>>>(n, g.t_comp, B, scale, Nk);
        e = cudaGetLastError();
    }
done:
    cudaFreeAsync(A, st);
    cudaFreeAsync(B, st);
    return e;
}

// Octant of the real-space tensor (for tests): out [6][N3][N2][N1], FP64.
cudaError_t newell_octant(int N1, int N2, int N3, double a, double b, double c, double *out, cudaStream_t st)
{
    TentRule tr = make_tent_rule();
    long nc = (long)N1 * N2 * N3;
    k_newell_octant<<<div_up(nc, 128), 128, 0, st>>>(N1, N2, N3, a, b, c, tr, out);
    return cudaGetLastError();
}

template cudaError_t build_tensor_spectrum<float>(const Geom &, double, double, double, const Cx<double> *, float *,
                                                  cudaStream_t);
template cudaError_t build_tensor_spectrum<double>(const Geom &, double, double, double, const Cx<double> *,
                                                   double *, cudaStream_t);

}  // namespace nm
