// Fused node kernel: exchange, uniaxial anisotropy, Zeeman and the cell->node demag average, divided
// by the lumped nodal mass (Eqs. weak_form_impl_f, weak_form_impl, mass_lumping), followed by the LLG
// right-hand side (Eq. llg) and the formation of the next Runge-Kutta stage input.
//
// Assembly by neighbour instead of by cell: node n couples to n + o (o in {-1,0,1}^3) through every
// cell that holds both nodes; those are the cells c = n - i with i_k = 1 where o_k = -1, i_k = 0
// where o_k = +1 and either where o_k = 0.  The element integral of such a pair depends only on the
// pattern d = |o|, so the variation at n is
//   dE_ex,n = sum_o Wex[d(o)] (sum_{cells} A_c) (m_{n+o} - m_n)         (rows of Kex sum to zero)
//   dE_an,n = -2 e sum_o Wm[d(o)] (sum_{cells} Ku_c) (e . m_{n+o})
// which is the cell-by-cell sum of the paper regrouped per neighbour (a gather, no atomics).
#include "local.cuh"

namespace nm {

template <typename T>
__device__ __forceinline__ double time_factor(double f, double ph, double t)
{
    return f == 0.0 ? 1.0 : sin(2.0 * 3.14159265358979323846 * f * t + ph);
}

// The node kernel walks a TX x TY tile of nodes along z.  Node planes of y (with a one-node halo in x
// and y) and cell planes of Ms_c H_c (the cells around the tile) rotate through shared memory: planes
// z-1, z, z+1 are read while plane z+2 (and cell plane z+1) are already being copied in with cp.async,
// so every value is read from global memory about once and the copies overlap the arithmetic.  Nodes
// and cells outside the mesh are filled with zeros (their weights are zero too).
constexpr int kTX = 32;
template <typename T>
constexpr int kTY = 4;  // 128-thread tiles, six FP32 blocks per SM at 80 registers (measured best of 32 x 2/4/8 tiles and 4-8 blocks)
constexpr int kNodeSlots = 4, kCellSlots = 3;

// a nodal or cell 3-vector
template <typename T>
struct V4 {
    T x, y, z;
};

// NS rotating planes of R x C 3-vectors in shared memory.  FP64: packed triples.  FP32: x and y as one
// 8-byte pair and z apart, 12 bytes per vector: a warp reads a row of vectors with one 8-byte and one
// 4-byte shared load, three wavefronts instead of the four of a 16-byte padded vector (the node
// kernel's shared-memory pipe is its busiest unit).
template <typename T, int NS, int R, int C>
struct Planes {
    V4<T> v[NS][R][C];
    __device__ __forceinline__ V4<T> get(int s, int r, int c) const { return v[s][r][c]; }
    __device__ __forceinline__ T *px(int s, int r, int c) { return &v[s][r][c].x; }
    __device__ __forceinline__ T *py(int s, int r, int c) { return &v[s][r][c].y; }
    __device__ __forceinline__ T *pz(int s, int r, int c) { return &v[s][r][c].z; }
    // element t of plane s in row-major order
    __device__ __forceinline__ T *px(int s, int t) { return &(&v[s][0][0])[t].x; }
    __device__ __forceinline__ T *py(int s, int t) { return &(&v[s][0][0])[t].y; }
    __device__ __forceinline__ T *pz(int s, int t) { return &(&v[s][0][0])[t].z; }
};
template <int NS, int R, int C>
struct Planes<float, NS, R, C> {
    float2 xy[NS][R][C];
    float z[NS][R][C];
    __device__ __forceinline__ V4<float> get(int s, int r, int c) const
    {
        const float2 a = xy[s][r][c];
        return V4<float>{a.x, a.y, z[s][r][c]};
    }
    __device__ __forceinline__ float *px(int s, int r, int c) { return &xy[s][r][c].x; }
    __device__ __forceinline__ float *py(int s, int r, int c) { return &xy[s][r][c].y; }
    __device__ __forceinline__ float *pz(int s, int r, int c) { return &z[s][r][c]; }
    __device__ __forceinline__ float *px(int s, int t) { return &(&xy[s][0][0])[t].x; }
    __device__ __forceinline__ float *py(int s, int t) { return &(&xy[s][0][0])[t].y; }
    __device__ __forceinline__ float *pz(int s, int t) { return &z[s][0][0] + t; }
};

template <typename T>
struct NodeSmem {
    static constexpr int SX = kTX + 2, SY = kTY<T> + 2;  // node plane with halo
    static constexpr int CX = kTX + 1, CY = kTY<T> + 1;  // cell plane around the tile
    Planes<T, kNodeSlots, SY, SX> y;  // node plane z in slot (z + 4) % 4
    Planes<T, kCellSlots, CY, CX> c;  // cell plane c3 in slot (c3 + 3) % 3, Ms_c H_c
    T hf[4];
};

// asynchronous copy of one value, or zero fill when !in
template <typename T>
__device__ __forceinline__ void cp_val(T *dst, const T *src, bool in)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = in ? (int)sizeof(T) : 0;
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}

// What one thread copies of every node plane: elements t = threadIdx.x and threadIdx.x + TX TY of the
// plane's row-major halo layout, each with its in-plane offset in the node array, or -1 where it lies
// outside the mesh (zero fill).  The same for every z: formed once per tile.
struct PlaneCopy {
    int node[2];
};

template <typename T>
__device__ __forceinline__ PlaneCopy plane_copy(const Geom &g, int x0, int y0)
{
    using S = NodeSmem<T>;
    constexpr int NT = kTX * kTY<T>;
    PlaneCopy pc;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int t = threadIdx.x + k * NT;
        const int r = t / S::SX, cc = t - r * S::SX;
        const int nx = x0 - 1 + cc, ny = y0 - 1 + r;
        pc.node[k] = (nx >= 0 && nx < g.nn1 && ny >= 0 && ny < g.nn2) ? ny * g.nn1 + nx : -1;
    }
    return pc;
}

template <typename T>
__device__ __forceinline__ void load_node_plane(const LocalParams<T> &p, const T *__restrict__ y, NodeSmem<T> &sm,
                                                int z, const PlaneCopy &pc)
{
    using S = NodeSmem<T>;
    constexpr int NT = kTX * kTY<T>;
    const Geom &g = p.g;
    const int sl = (z + kNodeSlots) % kNodeSlots;
    const bool zin = z >= 0 && z < g.nn3;
    const int ns = (int)g.ns, zo = z * g.nn2 * g.nn1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int t = threadIdx.x + k * NT;
        if (t < S::SX * S::SY) {
            const bool in = zin && pc.node[k] >= 0;
            const int n = in ? zo + pc.node[k] : 0;
            cp_val(sm.y.px(sl, t), y + n, in);
            cp_val(sm.y.py(sl, t), y + ns + n, in);
            cp_val(sm.y.pz(sl, t), y + 2 * ns + n, in);
        }
    }
}

template <typename T>
__device__ __forceinline__ void load_cell_plane(const LocalParams<T> &p, NodeSmem<T> &sm, int c3, int x0, int y0)
{
    using S = NodeSmem<T>;
    const Geom &g = p.g;
    if (!p.MsH || !(p.terms & NM_DEMAG)) return;  // the cell planes are not read
    const int sl = (c3 + kCellSlots) % kCellSlots;
    const bool zin = c3 >= 0 && c3 < g.N3;
    const int cs = (int)g.cs;
    for (int t = threadIdx.x; t < S::CX * S::CY; t += blockDim.x) {
        const int r = t / S::CX, cc = t - r * S::CX;
        const int c1 = x0 - 1 + cc, c2 = y0 - 1 + r;
        const bool in = zin && c1 >= 0 && c1 < g.N1 && c2 >= 0 && c2 < g.N2;
        const int c = in ? (c3 * g.N2 + c2) * g.N1 + c1 : 0;
        cp_val(sm.c.px(sl, r, cc), p.MsH + c, in);
        cp_val(sm.c.py(sl, r, cc), p.MsH + cs + c, in);
        cp_val(sm.c.pz(sl, r, cc), p.MsH + 2 * cs + c, in);
    }
}

template <typename T>
struct NodeField {
    T hx, hy, hz;
    T mx, my, mz;
    bool magnetic;
};

// Effective field at node (n1, n2, n3) = (x0 + tx, y0 + ty, z) from the shared planes.
//   MODE 1 (interior, uniform material): every cell around the node exists, the 27 assembled weights
//          are constants;
//   MODE 2 (uniform material, any node): the weight of an offset is the per-pattern constant times the
//          number of mesh cells holding both nodes, the product of per-axis counts;
//   MODE 0 (general): the weights are summed over the adjacent cells' material values.
template <typename T, int MODE>
__device__ __forceinline__ NodeField<T> node_field(const LocalParams<T> &p, const NodeSmem<T> &sm, int n1, int n2,
                                                   int n3, T im, int tx, int ty)
{
    const Geom &g = p.g;
    const int sz0 = (n3 + kNodeSlots) % kNodeSlots, szm = (n3 + kNodeSlots - 1) % kNodeSlots,
              szp = (n3 + 1) % kNodeSlots;
    const int cx0 = tx + 1, cy0 = ty + 1;
    NodeField<T> f;
    {
        const V4<T> m = sm.y.get(sz0, cy0, cx0);
        f.mx = m.x;
        f.my = m.y;
        f.mz = m.z;
    }
    f.magnetic = im > T(0);
    T ex = 0, ey = 0, ez = 0, pe = 0;
    if (MODE == 1) {
        // sum_o w_o (m_{n+o} - m_n) = sum_{o != 0} w_o m_{n+o} - (sum w) m_n;  anisotropy: sum_o c_o m_{n+o}
        T sx = 0, sy = 0, sz = 0, ax = 0, ay = 0, az = 0;
#pragma unroll
        for (int o3 = -1; o3 <= 1; ++o3) {
            const int slot = o3 < 0 ? szm : (o3 > 0 ? szp : sz0);
#pragma unroll
            for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
                for (int o1 = -1; o1 <= 1; ++o1) {
                    const int k = (o3 + 1) * 9 + (o2 + 1) * 3 + (o1 + 1);
                    const V4<T> q = sm.y.get(slot, cy0 + o2, cx0 + o1);
                    if (k != 13) {
                        sx += p.wex27[k] * q.x;
                        sy += p.wex27[k] * q.y;
                        sz += p.wex27[k] * q.z;
                    }
                    ax += p.wan27[k] * q.x;
                    ay += p.wan27[k] * q.y;
                    az += p.wan27[k] * q.z;
                }
        }
        ex = sx - p.wex_sum * f.mx;
        ey = sy - p.wex_sum * f.my;
        ez = sz - p.wex_sum * f.mz;
        pe = p.e0 * ax + p.e1 * ay + p.e2 * az;
    } else if (MODE == 2) {
        // cells n_k - 1 (pattern i_k = 1) and n_k (i_k = 0) along each axis
        const int cm1 = n1 >= 1 && n1 - 1 < g.N1, cp1 = n1 < g.N1;
        const int cm2 = n2 >= 1 && n2 - 1 < g.N2, cp2 = n2 < g.N2;
        const int cm3 = n3 >= 1 && n3 - 1 < g.N3, cp3 = n3 < g.N3;
        T sx = 0, sy = 0, sz = 0, ax = 0, ay = 0, az = 0, wsum = 0;
#pragma unroll
        for (int o3 = -1; o3 <= 1; ++o3) {
            const int slot = o3 < 0 ? szm : (o3 > 0 ? szp : sz0);
            const int k3 = o3 < 0 ? cm3 : (o3 > 0 ? cp3 : cm3 + cp3);
#pragma unroll
            for (int o2 = -1; o2 <= 1; ++o2) {
                const int k23 = k3 * (o2 < 0 ? cm2 : (o2 > 0 ? cp2 : cm2 + cp2));
#pragma unroll
                for (int o1 = -1; o1 <= 1; ++o1) {
                    const int cnt = k23 * (o1 < 0 ? cm1 : (o1 > 0 ? cp1 : cm1 + cp1));
                    const int d = ((o1 != 0) << 2) | ((o2 != 0) << 1) | (o3 != 0);
                    const T fc = (T)cnt;
                    const V4<T> q = sm.y.get(slot, cy0 + o2, cx0 + o1);
                    if (d != 0) {
                        const T w = p.wexd[d] * fc;
                        sx += w * q.x;
                        sy += w * q.y;
                        sz += w * q.z;
                        wsum += w;
                    }
                    const T wa = p.wand[d] * fc;
                    ax += wa * q.x;
                    ay += wa * q.y;
                    az += wa * q.z;
                }
            }
        }
        ex = sx - wsum * f.mx;
        ey = sy - wsum * f.my;
        ez = sz - wsum * f.mz;
        pe = p.e0 * ax + p.e1 * ay + p.e2 * az;
    } else {
        T a[8], ku[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c1 = n1 - ((i >> 2) & 1), c2 = n2 - ((i >> 1) & 1), c3 = n3 - (i & 1);
            const bool valid = c1 >= 0 && c1 < g.N1 && c2 >= 0 && c2 < g.N2 && c3 >= 0 && c3 < g.N3;
            const int c = valid ? (c3 * g.N2 + c2) * g.N1 + c1 : 0;
            const T Ms = valid ? (p.Ms ? p.Ms[c] : p.Ms0) : T(0);
            const bool mag = valid && Ms > T(0);
            a[i] = (mag && (p.terms & NM_EXCH)) ? (p.A ? p.A[c] : p.A0) : T(0);
            ku[i] = (mag && (p.terms & NM_ANIS)) ? (p.Ku ? p.Ku[c] : p.Ku0) : T(0);
        }
#pragma unroll
        for (int o3 = -1; o3 <= 1; ++o3) {
            const int slot = o3 < 0 ? szm : (o3 > 0 ? szp : sz0);
#pragma unroll
            for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
                for (int o1 = -1; o1 <= 1; ++o1) {
                    T S = 0, K = 0;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int i1 = (i >> 2) & 1, i2 = (i >> 1) & 1, i3 = i & 1;
                        const bool comp = (o1 == -1 ? i1 == 1 : (o1 == 1 ? i1 == 0 : true)) &&
                                          (o2 == -1 ? i2 == 1 : (o2 == 1 ? i2 == 0 : true)) &&
                                          (o3 == -1 ? i3 == 1 : (o3 == 1 ? i3 == 0 : true));
                        if (comp) {
                            S += a[i];
                            K += ku[i];
                        }
                    }
                    const int d = ((o1 != 0) << 2) | ((o2 != 0) << 1) | (o3 != 0);
                    const bool self = (o1 == 0 && o2 == 0 && o3 == 0);
                    const V4<T> q = sm.y.get(slot, cy0 + o2, cx0 + o1);
                    if (!self) {
                        const T w = p.Wex[d] * S;
                        ex += w * (q.x - f.mx);
                        ey += w * (q.y - f.my);
                        ez += w * (q.z - f.mz);
                    }
                    pe += p.Wm[d] * K * (p.e0 * q.x + p.e1 * q.y + p.e2 * q.z);
                }
        }
    }
    // -dE / mass: exchange and anisotropy
    T hx = -ex + T(2) * p.e0 * pe;
    T hy = -ey + T(2) * p.e1 * pe;
    T hz = -ez + T(2) * p.e2 * pe;
    // cell -> node: demag (Ms_c H_c, from the shared cell planes) and cell applied field (Ms_c h_c)
    T cx_ = 0, cy_ = 0, cz_ = 0;
    if (p.MsH && (p.terms & NM_DEMAG)) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int i1 = (i >> 2) & 1, i2 = (i >> 1) & 1, i3 = i & 1;
            const V4<T> v = sm.c.get((n3 - i3 + kCellSlots) % kCellSlots, cy0 - i2, cx0 - i1);
            cx_ += v.x;
            cy_ += v.y;
            cz_ += v.z;
        }
    }
    if (p.Msh && (p.terms & NM_ZEE)) {
        const T sc = sm.hf[3];
        const long cs = g.cs;
        T ax = 0, ay = 0, az = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c1 = n1 - ((i >> 2) & 1), c2 = n2 - ((i >> 1) & 1), c3 = n3 - (i & 1);
            if (c1 >= 0 && c1 < g.N1 && c2 >= 0 && c2 < g.N2 && c3 >= 0 && c3 < g.N3) {
                const int c = (c3 * g.N2 + c2) * g.N1 + c1;
                ax += p.Msh[c];
                ay += p.Msh[cs + c];
                az += p.Msh[2 * cs + c];
            }
        }
        cx_ += sc * ax;
        cy_ += sc * ay;
        cz_ += sc * az;
    }
    if (p.raw) {
        // -dE itself (the transpose products of the adjoint): no lumped-mass division
        f.hx = hx + p.mu0V8 * cx_;
        f.hy = hy + p.mu0V8 * cy_;
        f.hz = hz + p.mu0V8 * cz_;
        return f;
    }
    hx = im * (hx + p.mu0V8 * cx_);
    hy = im * (hy + p.mu0V8 * cy_);
    hz = im * (hz + p.mu0V8 * cz_);
    if (f.magnetic && (p.terms & NM_ZEE)) {
        hx += sm.hf[0];
        hy += sm.hf[1];
        hz += sm.hf[2];
    }
    f.hx = hx; f.hy = hy; f.hz = hz;
    return f;
}

// FP32 stage kernels that form the next stage input from three or more earlier slopes stage each node's
// own values one plane ahead in shared memory, beside the node and cell planes: 1/mass, the earlier
// slopes with non-zero coefficients and the FP32 copy of m.  Their global loads then have a whole plane
// of work to arrive in, instead of stalling the stage-input sums (with fewer slopes the extra copies
// cost more than the stalls they remove).  Every Runge-Kutta tableau of the library has at most
// kOwnSlopes such slopes per stage.
constexpr int kOwnSlopes = 4, kOwnVals = 1 + 3 * kOwnSlopes + 3;

// Blocks of a node launch (1D grid): blocks b < full walk tile b over all node planes; the tiles after
// them (the ones that would otherwise run alone in a last partial wave of long blocks) are split along z
// into `chunks` blocks of zc planes each.  Tile t covers nodes x0 = (t % bxn) TX, y0 = (t / bxn) TY.
struct NodeGrid {
    int bxn, full, chunks, zc;
};

// STAGE = false: write H (effective-field evaluation); true: write the LLG slope k_s and the next stage
// input.  Each block covers nodes x0.. x0+TX-1, y0.. y0+TY-1 and z in [z0, z1) (NodeGrid).
// OWN (FP32 stage kernels with a next stage input from the FP32 copy of m and at most kOwnSlopes
// earlier slopes): the node's own values are staged in shared memory.
template <typename T, bool STAGE, bool DMI = false, bool OWN = false>
__global__ void __launch_bounds__(kTX *kTY<T>, sizeof(T) == 4 ? 6 : 3) k_node(LocalParams<T> p, const T *__restrict__ y,
                                                        T *__restrict__ out, T *__restrict__ y_next, StageArgs sa,
                                                        double t_heff, NodeGrid ng)
{
    static_assert(!OWN || (sizeof(T) == 4 && STAGE && !DMI), "own-value staging is for FP32 stage kernels");
    if (STAGE && sa.ctl && sa.ctl->done) return;
    constexpr int TY = kTY<T>;
    __shared__ NodeSmem<T> sm;
    __shared__ float own_sm[OWN ? 2 : 1][OWN ? kOwnVals : 1][TY][kTX];
    const Geom &g = p.g;
    const int b = blockIdx.x, split = b >= ng.full;
    const int tile = split ? ng.full + (b - ng.full) / ng.chunks : b;
    const int z0 = split ? (b - ng.full) % ng.chunks * ng.zc : 0, z1 = split ? min(g.nn3, z0 + ng.zc) : g.nn3;
    const int x0 = tile % ng.bxn * kTX, y0 = tile / ng.bxn * TY;
    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    const int n1 = x0 + tx, n2 = y0 + ty;
    const bool active = n1 < g.nn1 && n2 < g.nn2;
    // OWN: copy node plane zz's own values of this thread into slot zz & 1
    auto load_own = [&](int zz) {
        if constexpr (OWN) {
            const int nq = (zz * g.nn2 + n2) * g.nn1 + n1, nsq = (int)g.ns;
            float(*o)[TY][kTX] = own_sm[zz & 1];
            cp_val(&o[0][ty][tx], (const float *)p.inv_mass + nq, true);
            int q = 1;
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                if (j + 1 >= sa.s) break;
                if (sa.af[j] == 0.f) continue;
                const float *kj = (const float *)sa.k[j];
                cp_val(&o[q][ty][tx], kj + nq, true);
                cp_val(&o[q + 1][ty][tx], kj + nsq + nq, true);
                cp_val(&o[q + 2][ty][tx], kj + 2 * nsq + nq, true);
                q += 3;
            }
            cp_val(&o[kOwnVals - 3][ty][tx], sa.mf + nq, true);
            cp_val(&o[kOwnVals - 2][ty][tx], sa.mf + nsq + nq, true);
            cp_val(&o[kOwnVals - 1][ty][tx], sa.mf + 2 * nsq + nq, true);
        }
    };
    if (threadIdx.x == 0) {
        const double t = STAGE ? (sa.ctl ? sa.ctl->t + sa.c_s * sa.ctl->dt : sa.t_fixed) : t_heff;
        const double su = time_factor<T>(p.hu_freq, p.hu_phase, t);
        sm.hf[0] = (T)(p.hu0 * su);
        sm.hf[1] = (T)(p.hu1 * su);
        sm.hf[2] = (T)(p.hu2 * su);
        sm.hf[3] = (T)time_factor<T>(p.hc_freq, p.hc_phase, t);
    }
    const PlaneCopy pc = plane_copy<T>(g, x0, y0);
    // copy groups: {node z0-1, node z0, cell z0-1}, then per z the group {node z+1, cell z}
    load_node_plane(p, y, sm, z0 - 1, pc);
    load_node_plane(p, y, sm, z0, pc);
    load_cell_plane(p, sm, z0 - 1, x0, y0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    load_node_plane(p, y, sm, z0 + 1, pc);
    load_cell_plane(p, sm, z0, x0, y0);
    if (OWN && active) load_own(z0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const int ns = (int)g.ns;
    double dt = 0.0;
    if (STAGE) dt = sa.ctl ? sa.ctl->dt : 0.0;
    const float dtf = (float)dt;
    // the tile's x-y footprint has all eight cells around every node (uniform material)
    const bool tile_inner = p.uniform && x0 >= 1 && x0 + kTX <= g.N1 && y0 >= 1 && y0 + TY <= g.N2;
    for (int z = z0; z < z1; ++z) {
        // start the copies for the next plane (into the slots of planes z - 2 and cells z - 2, free since
        // the barrier that ended the previous iteration), then wait for everything but them
        if (z + 1 < z1) {
            load_node_plane(p, y, sm, z + 2, pc);
            load_cell_plane(p, sm, z + 1, x0, y0);
            if (OWN && active) load_own(z + 1);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        // this node's own values (1/mass; for the next stage input, the earlier slopes and the FP32 copy
        // of m) do not depend on the shared planes: their loads are issued before the wait and barrier
        const int n = (z * g.nn2 + n2) * g.nn1 + n1;
        T im = T(0), px = 0, py = 0, pz = 0;
        float mfx = 0.f, mfy = 0.f, mfz = 0.f;
        T dmx = 0, dmy = 0, dmz = 0;  // raw DMI field of this node (DMI instances)
        if (DMI && active) {
            dmx = p.hdmi[n];
            dmy = p.hdmi[ns + n];
            dmz = p.hdmi[2 * ns + n];
        }
        if (!OWN && active) {
            im = p.inv_mass[n];
            if (STAGE && y_next) {
#pragma unroll
                for (int j = 0; j < 7; ++j) {
                    if (j + 1 >= sa.s) break;
                    const T aj = sizeof(T) == 4 ? (T)sa.af[j] : (T)sa.a[j];
                    if (aj == T(0)) continue;
                    const T *kj = (const T *)sa.k[j];
                    px += aj * kj[n];
                    py += aj * kj[ns + n];
                    pz += aj * kj[2 * ns + n];
                }
                if (sizeof(T) == 4 && sa.mf) {
                    mfx = sa.mf[n];
                    mfy = sa.mf[ns + n];
                    mfz = sa.mf[2 * ns + n];
                }
            }
        }
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        const bool interior = tile_inner && z >= 1 && z <= g.N3 - 1;
        if constexpr (OWN) {
            if (active) im = (T)own_sm[z & 1][0][ty][tx];
        }
        if (active) {
            NodeField<T> f = interior    ? node_field<T, 1>(p, sm, n1, n2, z, im, tx, ty)
                             : p.uniform ? node_field<T, 2>(p, sm, n1, n2, z, im, tx, ty)
                                         : node_field<T, 0>(p, sm, n1, n2, z, im, tx, ty);
            if (DMI) {
                const T sc = p.raw ? T(1) : im;
                f.hx += sc * dmx;
                f.hy += sc * dmy;
                f.hz += sc * dmz;
            }
            if (!STAGE) {
                out[n] = f.hx;
                out[ns + n] = f.hy;
                out[2 * ns + n] = f.hz;
            } else {
                T kx = 0, ky = 0, kz = 0;
                if (f.magnetic) {
                    // k = -gamma'(m x H + alpha m x (m x H))
                    const T ax = f.my * f.hz - f.mz * f.hy;
                    const T ay = f.mz * f.hx - f.mx * f.hz;
                    const T az = f.mx * f.hy - f.my * f.hx;
                    const T bx = f.my * az - f.mz * ay;
                    const T by = f.mz * ax - f.mx * az;
                    const T bz = f.mx * ay - f.my * ax;
                    const T gm = p.gam_t, al = p.alpha_t;
                    kx = -gm * (ax + al * bx);
                    ky = -gm * (ay + al * by);
                    kz = -gm * (az + al * bz);
                }
                out[n] = kx;
                out[ns + n] = ky;
                out[2 * ns + n] = kz;
                if (y_next) {
                    // y_{s+1} = m + dt sum_{j<=s} a_{s+1,j} k_j: the slope combination in the working
                    // precision
                    if constexpr (OWN) {
                        // the earlier slopes and the FP32 copy of m from the staged own values
                        const float(*o)[TY][kTX] = own_sm[z & 1];
                        int q = 1;
#pragma unroll
                        for (int j = 0; j < 7; ++j) {
                            if (j + 1 >= sa.s) break;
                            const float aj = sa.af[j];
                            if (aj == 0.f) continue;
                            px += aj * o[q][ty][tx];
                            py += aj * o[q + 1][ty][tx];
                            pz += aj * o[q + 2][ty][tx];
                            q += 3;
                        }
                        mfx = o[kOwnVals - 3][ty][tx];
                        mfy = o[kOwnVals - 2][ty][tx];
                        mfz = o[kOwnVals - 1][ty][tx];
                    }
                    const T as = sizeof(T) == 4 ? (T)sa.af_s : (T)sa.a_s;
                    const T ax = px + as * kx, ay = py + as * ky, az = pz + as * kz;
                    if (sizeof(T) == 4 && sa.mf) {
                        // FP32 path: y_{s+1} is an FP32 quantity, formed from the FP32 copy of m
                        y_next[n] = (T)(mfx + dtf * (float)ax);
                        y_next[ns + n] = (T)(mfy + dtf * (float)ay);
                        y_next[2 * ns + n] = (T)(mfz + dtf * (float)az);
                    } else {
                        y_next[n] = (T)(sa.m[n] + dt * (double)ax);
                        y_next[ns + n] = (T)(sa.m[ns + n] + dt * (double)ay);
                        y_next[2 * ns + n] = (T)(sa.m[2 * ns + n] + dt * (double)az);
                    }
                }
            }
        }
        __syncthreads();  // the next iteration overwrites the slots of planes z - 1 and c3 = z - 1
    }
}

// 2D basis (section "Low-Dimensional Geometries"): one node layer; the basis function of node (n1, n2)
// is constant along z over all N3 cell layers, so it couples to the 9 nodes n + o (o in {-1,0,1}^2)
// through the in-plane cells holding both nodes, in every layer.  With per-layer pattern integrals
// Wex2, Wm2 (d = 2|o1| + |o2|) the variation at n is
//   dE_ex = sum_o Wex2[d] (sum_{cells} A_c) (m_{n+o} - m_n),  dE_an = -2 e sum_o Wm2[d] (sum Ku_c) (e . m_{n+o})
// and the cell->node average takes Ms_c H_c over the 4 in-plane cells of every layer with weight
// mu0 V/4.  One thread per node; neighbours and cells are read through L1 (thin films: N3 is small).
template <typename T, bool STAGE>
__global__ void __launch_bounds__(256) k_node2d(LocalParams<T> p, const T *__restrict__ y, T *__restrict__ out,
                                                T *__restrict__ y_next, StageArgs sa, double t_heff)
{
    if (STAGE && sa.ctl && sa.ctl->done) return;
    const Geom &g = p.g;
    const int n1 = blockIdx.x * 32 + (threadIdx.x & 31), n2 = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (n1 >= g.nn1 || n2 >= g.nn2) return;
    const int ns = (int)g.ns, n = n2 * g.nn1 + n1;
    const double t = STAGE ? (sa.ctl ? sa.ctl->t + sa.c_s * sa.ctl->dt : sa.t_fixed) : t_heff;
    const T im = p.inv_mass[n];
    const bool magnetic = im > T(0);
    // per in-plane cell (i1, i2): layer sums of A, Ku over magnetic cells, of Ms_c H_c and of Ms_c h_c
    T SA[4], SK[4];
    T cx = 0, cy = 0, cz = 0, zx = 0, zy = 0, zz = 0;
    const bool demag = p.MsH && (p.terms & NM_DEMAG), zee_c = p.Msh && (p.terms & NM_ZEE);
    const long cs = g.cs;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        SA[i] = T(0);
        SK[i] = T(0);
        const int c1 = n1 - ((i >> 1) & 1), c2 = n2 - (i & 1);
        if (c1 < 0 || c1 >= g.N1 || c2 < 0 || c2 >= g.N2) continue;
        for (int c3 = 0; c3 < g.N3; ++c3) {
            const int c = (c3 * g.N2 + c2) * g.N1 + c1;
            const T Ms = p.Ms ? p.Ms[c] : p.Ms0;
            if (!(Ms > T(0))) continue;
            if (p.terms & NM_EXCH) SA[i] += p.A ? p.A[c] : p.A0;
            if (p.terms & NM_ANIS) SK[i] += p.Ku ? p.Ku[c] : p.Ku0;
            if (demag) {
                cx += p.MsH[c];
                cy += p.MsH[cs + c];
                cz += p.MsH[2 * cs + c];
            }
            if (zee_c) {
                zx += p.Msh[c];
                zy += p.Msh[cs + c];
                zz += p.Msh[2 * cs + c];
            }
        }
    }
    const T mx = y[n], my = y[ns + n], mz = y[2 * ns + n];
    T ex = 0, ey = 0, ez = 0, pe = 0;
#pragma unroll
    for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
        for (int o1 = -1; o1 <= 1; ++o1) {
            // in-plane cells holding both n and n + o: i_k = 1 where o_k = -1, 0 where o_k = +1, either at 0
            T S = 0, K = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int i1 = (i >> 1) & 1, i2 = i & 1;
                if ((o1 == -1 && i1 != 1) || (o1 == 1 && i1 != 0) || (o2 == -1 && i2 != 1) || (o2 == 1 && i2 != 0))
                    continue;
                S += SA[i];
                K += SK[i];
            }
            const int d = 2 * (o1 != 0) + (o2 != 0);
            const int q1 = n1 + o1, q2 = n2 + o2;
            if (q1 < 0 || q1 >= g.nn1 || q2 < 0 || q2 >= g.nn2) continue;  // (its weights are zero)
            const int q = q2 * g.nn1 + q1;
            const T qx = y[q], qy = y[ns + q], qz = y[2 * ns + q];
            if (o1 != 0 || o2 != 0) {
                const T w = p.Wex2[d] * S;
                ex += w * (qx - mx);
                ey += w * (qy - my);
                ez += w * (qz - mz);
            }
            pe += p.Wm2[d] * K * (p.e0 * qx + p.e1 * qy + p.e2 * qz);
        }
    T hx = -ex + T(2) * p.e0 * pe, hy = -ey + T(2) * p.e1 * pe, hz = -ez + T(2) * p.e2 * pe;
    if (zee_c) {
        const T sc = (T)time_factor<T>(p.hc_freq, p.hc_phase, t);
        cx += sc * zx;
        cy += sc * zy;
        cz += sc * zz;
    }
    if (p.raw) {
        hx += p.mu0V4 * cx;
        hy += p.mu0V4 * cy;
        hz += p.mu0V4 * cz;
    } else {
        hx = im * (hx + p.mu0V4 * cx);
        hy = im * (hy + p.mu0V4 * cy);
        hz = im * (hz + p.mu0V4 * cz);
        if (magnetic && (p.terms & NM_ZEE)) {
            const T su = (T)time_factor<T>(p.hu_freq, p.hu_phase, t);
            hx += (T)p.hu0 * su;
            hy += (T)p.hu1 * su;
            hz += (T)p.hu2 * su;
        }
    }
    if (!STAGE) {
        out[n] = hx;
        out[ns + n] = hy;
        out[2 * ns + n] = hz;
        return;
    }
    T kx = 0, ky = 0, kz = 0;
    if (magnetic) {
        const T ax = my * hz - mz * hy, ay = mz * hx - mx * hz, az = mx * hy - my * hx;
        const T bx = my * az - mz * ay, by = mz * ax - mx * az, bz = mx * ay - my * ax;
        kx = -p.gam_t * (ax + p.alpha_t * bx);
        ky = -p.gam_t * (ay + p.alpha_t * by);
        kz = -p.gam_t * (az + p.alpha_t * bz);
    }
    out[n] = kx;
    out[ns + n] = ky;
    out[2 * ns + n] = kz;
    if (y_next) {
        T px = 0, py = 0, pz = 0;
        for (int j = 0; j + 1 < sa.s && j < 7; ++j) {
            const T aj = sizeof(T) == 4 ? (T)sa.af[j] : (T)sa.a[j];
            if (aj == T(0)) continue;
            const T *kj = (const T *)sa.k[j];
            px += aj * kj[n];
            py += aj * kj[ns + n];
            pz += aj * kj[2 * ns + n];
        }
        const T as = sizeof(T) == 4 ? (T)sa.af_s : (T)sa.a_s;
        px += as * kx;
        py += as * ky;
        pz += as * kz;
        const double dt = sa.ctl ? sa.ctl->dt : 0.0;
        if (sizeof(T) == 4 && sa.mf) {
            const float dtf = (float)dt;
            y_next[n] = (T)(sa.mf[n] + dtf * (float)px);
            y_next[ns + n] = (T)(sa.mf[ns + n] + dtf * (float)py);
            y_next[2 * ns + n] = (T)(sa.mf[2 * ns + n] + dtf * (float)pz);
        } else {
            y_next[n] = (T)(sa.m[n] + dt * (double)px);
            y_next[ns + n] = (T)(sa.m[ns + n] + dt * (double)py);
            y_next[2 * ns + n] = (T)(sa.m[2 * ns + n] + dt * (double)pz);
        }
    }
}

// 1D basis (section "Low-Dimensional Geometries"): nodes along x only; the basis function of node n1 is
// the hat function of x, constant over the whole N2 x N3 cross-section, so it couples to n1 - 1 and
// n1 + 1 through the cells of the slab between them (c1 = n1 - 1 on the left, c1 = n1 on the right).
// With per-cell pattern integrals Wex1, Wm1 (d = |o1|) and slab sums S_o of A, K_o of Ku over magnetic
// cells,
//   dE_ex = sum_{o = -1, 1} Wex1[1] S_o (m_{n+o} - m_n),
//   dE_an = -2 e [Wm1[0] (K_-1 + K_1) (e . m_n) + sum_{o = -1, 1} Wm1[1] K_o (e . m_{n+o})],
// and the cell->node average takes Ms_c H_c over the cells of both slabs with weight mu0 V/2.  One block
// per node: its threads sum the slab cells in a fixed order and tree, thread 0 finishes the node.
constexpr int kNode1dThreads = 128;

template <typename T, bool STAGE>
__global__ void __launch_bounds__(kNode1dThreads) k_node1d(LocalParams<T> p, const T *__restrict__ y,
                                                           T *__restrict__ out, T *__restrict__ y_next, StageArgs sa,
                                                           double t_heff)
{
    if (STAGE && sa.ctl && sa.ctl->done) return;
    const Geom &g = p.g;
    const int n1 = blockIdx.x;
    // v: slab sums of A (left, right), of Ku (left, right), of Ms_c H_c (3) and of Ms_c h_c (3)
    constexpr int NV = 10;
    T v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = T(0);
    const bool demag = p.MsH && (p.terms & NM_DEMAG), zee_c = p.Msh && (p.terms & NM_ZEE);
    const long cs = g.cs;
    const int ncs = g.N2 * g.N3;
    for (int s = 0; s < 2; ++s) {
        const int c1 = n1 - 1 + s;
        if (c1 < 0 || c1 >= g.N1) continue;
        for (int j = threadIdx.x; j < ncs; j += blockDim.x) {
            const long c = (long)j * g.N1 + c1;  // cell (c1, j mod N2, j div N2)
            const T Ms = p.Ms ? p.Ms[c] : p.Ms0;
            if (!(Ms > T(0))) continue;
            if (p.terms & NM_EXCH) v[s] += p.A ? p.A[c] : p.A0;
            if (p.terms & NM_ANIS) v[2 + s] += p.Ku ? p.Ku[c] : p.Ku0;
            if (demag) {
                v[4] += p.MsH[c];
                v[5] += p.MsH[cs + c];
                v[6] += p.MsH[2 * cs + c];
            }
            if (zee_c) {
                v[7] += p.Msh[c];
                v[8] += p.Msh[cs + c];
                v[9] += p.Msh[2 * cs + c];
            }
        }
    }
    __shared__ T red[kNode1dThreads / 32][NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        T x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[w][i] = x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        T x = T(0);
        for (int k = 0; k < kNode1dThreads / 32; ++k) x += red[k][i];
        v[i] = x;
    }
    const int ns = (int)g.ns, n = n1;
    const double t = STAGE ? (sa.ctl ? sa.ctl->t + sa.c_s * sa.ctl->dt : sa.t_fixed) : t_heff;
    const T im = p.inv_mass[n];
    const bool magnetic = im > T(0);
    const T mx = y[n], my = y[ns + n], mz = y[2 * ns + n];
    T ex = 0, ey = 0, ez = 0;
    T pe = p.Wm1[0] * (v[2] + v[3]) * (p.e0 * mx + p.e1 * my + p.e2 * mz);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int q = s == 0 ? n1 - 1 : n1 + 1;
        if (q < 0 || q >= g.nn1) continue;  // (its slab does not exist)
        const T qx = y[q], qy = y[ns + q], qz = y[2 * ns + q];
        const T wq = p.Wex1[1] * v[s];
        ex += wq * (qx - mx);
        ey += wq * (qy - my);
        ez += wq * (qz - mz);
        pe += p.Wm1[1] * v[2 + s] * (p.e0 * qx + p.e1 * qy + p.e2 * qz);
    }
    T hx = -ex + T(2) * p.e0 * pe, hy = -ey + T(2) * p.e1 * pe, hz = -ez + T(2) * p.e2 * pe;
    T cx = v[4], cy = v[5], cz = v[6];
    if (zee_c) {
        const T sc = (T)time_factor<T>(p.hc_freq, p.hc_phase, t);
        cx += sc * v[7];
        cy += sc * v[8];
        cz += sc * v[9];
    }
    if (p.raw) {
        hx += p.mu0V2 * cx;
        hy += p.mu0V2 * cy;
        hz += p.mu0V2 * cz;
    } else {
        hx = im * (hx + p.mu0V2 * cx);
        hy = im * (hy + p.mu0V2 * cy);
        hz = im * (hz + p.mu0V2 * cz);
        if (magnetic && (p.terms & NM_ZEE)) {
            const T su = (T)time_factor<T>(p.hu_freq, p.hu_phase, t);
            hx += (T)p.hu0 * su;
            hy += (T)p.hu1 * su;
            hz += (T)p.hu2 * su;
        }
    }
    if (!STAGE) {
        out[n] = hx;
        out[ns + n] = hy;
        out[2 * ns + n] = hz;
        return;
    }
    T kx = 0, ky = 0, kz = 0;
    if (magnetic) {
        const T ax = my * hz - mz * hy, ay = mz * hx - mx * hz, az = mx * hy - my * hx;
        const T bx = my * az - mz * ay, by = mz * ax - mx * az, bz = mx * ay - my * ax;
        kx = -p.gam_t * (ax + p.alpha_t * bx);
        ky = -p.gam_t * (ay + p.alpha_t * by);
        kz = -p.gam_t * (az + p.alpha_t * bz);
    }
    out[n] = kx;
    out[ns + n] = ky;
    out[2 * ns + n] = kz;
    if (y_next) {
        T px = 0, py = 0, pz = 0;
        for (int j = 0; j + 1 < sa.s && j < 7; ++j) {
            const T aj = sizeof(T) == 4 ? (T)sa.af[j] : (T)sa.a[j];
            if (aj == T(0)) continue;
            const T *kj = (const T *)sa.k[j];
            px += aj * kj[n];
            py += aj * kj[ns + n];
            pz += aj * kj[2 * ns + n];
        }
        const T as = sizeof(T) == 4 ? (T)sa.af_s : (T)sa.a_s;
        px += as * kx;
        py += as * ky;
        pz += as * kz;
        const double dt = sa.ctl ? sa.ctl->dt : 0.0;
        if (sizeof(T) == 4 && sa.mf) {
            const float dtf = (float)dt;
            y_next[n] = (T)(sa.mf[n] + dtf * (float)px);
            y_next[ns + n] = (T)(sa.mf[ns + n] + dtf * (float)py);
            y_next[2 * ns + n] = (T)(sa.mf[2 * ns + n] + dtf * (float)pz);
        } else {
            y_next[n] = (T)(sa.m[n] + dt * (double)px);
            y_next[ns + n] = (T)(sa.m[ns + n] + dt * (double)py);
            y_next[2 * ns + n] = (T)(sa.m[2 * ns + n] + dt * (double)pz);
        }
    }
}

// Interfacial DMI, E = int D [m_z div m - (m . grad) m_z] (a reading of the paper's "antisymmetric
// exchange"), assembled like the exchange: with G_k(i,i') = int_cell phi_i d_k phi_i' and its
// antisymmetric part A_k, node n couples to n + o through every magnetic cell holding both nodes,
//   A_x(n, n+o) = o1 (mass integrals along y, z of the pattern),  A_y(n, n+o) = o2 (along x, z),
//   dE_x = -sum_o S_o A_x m_{n+o,z},  dE_y = -sum_o S_o A_y m_{n+o,z},
//   dE_z = sum_o S_o (A_x m_{n+o,x} + A_y m_{n+o,y}),        S_o = sum_{cells} D_c.
// Writes the raw field -dE per node (the node kernel scales it by 1/mass).  One thread per node,
// neighbours through L1.
template <typename T>
__global__ void __launch_bounds__(256) k_dmi(LocalParams<T> p, const T *__restrict__ y, T *__restrict__ out)
{
    const Geom &g = p.g;
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= g.n_nodes) return;
    const int n1 = (int)(n % g.nn1);
    const long r = n / g.nn1;
    const int n2 = (int)(r % g.nn2), n3 = (int)(r / g.nn2);
    const long ns = g.ns;
    T Dc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c1 = n1 - ((i >> 2) & 1), c2 = n2 - ((i >> 1) & 1), c3 = n3 - (i & 1);
        const bool valid = c1 >= 0 && c1 < g.N1 && c2 >= 0 && c2 < g.N2 && c3 >= 0 && c3 < g.N3;
        const int c = valid ? (c3 * g.N2 + c2) * g.N1 + c1 : 0;
        const T Ms = valid ? (p.Ms ? p.Ms[c] : p.Ms0) : T(0);
        Dc[i] = (valid && Ms > T(0)) ? (p.Dm ? p.Dm[c] : p.D0) : T(0);
    }
    T ex = 0, ey = 0, ez = 0;
#pragma unroll
    for (int o3 = -1; o3 <= 1; ++o3)
#pragma unroll
        for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
            for (int o1 = -1; o1 <= 1; ++o1) {
                if (o1 == 0 && o2 == 0) continue;  // no in-plane derivative couples them
                T S = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int i1 = (i >> 2) & 1, i2 = (i >> 1) & 1, i3 = i & 1;
                    const bool both = (o1 == -1 ? i1 == 1 : (o1 == 1 ? i1 == 0 : true)) &&
                                      (o2 == -1 ? i2 == 1 : (o2 == 1 ? i2 == 0 : true)) &&
                                      (o3 == -1 ? i3 == 1 : (o3 == 1 ? i3 == 0 : true));
                    if (both) S += Dc[i];
                }
                const int q1 = n1 + o1, q2 = n2 + o2, q3 = n3 + o3;
                if (q1 < 0 || q1 >= g.nn1 || q2 < 0 || q2 >= g.nn2 || q3 < 0 || q3 >= g.nn3) continue;
                const long q = ((long)q3 * g.nn2 + q2) * g.nn1 + q1;
                const T ax = o1 == 0 ? T(0) : T(o1) * p.dmx[2 * (o2 != 0) + (o3 != 0)] * S;
                const T ay = o2 == 0 ? T(0) : T(o2) * p.dmy[2 * (o1 != 0) + (o3 != 0)] * S;
                const T qx = y[q], qy = y[ns + q], qz = y[2 * ns + q];
                ex += -ax * qz;
                ey += -ay * qz;
                ez += ax * qx + ay * qy;
            }
    out[n] = -ex;
    out[ns + n] = -ey;
    out[2 * ns + n] = -ez;
}

// Launch shape of a node kernel instance.  R = blocks the device holds at once (occupancy times SMs,
// queried once per instance).  With T tiles, the first T - (T mod R) tiles make whole waves of full-depth
// blocks; the remaining T mod R tiles are split along z into about R / (T mod R) chunks each, so that
// the last wave is short instead of a full-length wave on a fraction of the SMs.  Fewer tiles than R:
// every tile is split the same way.
template <typename T, bool STAGE, bool DMI, bool OWN = false>
static NodeGrid node_grid(const Geom &g, int *blocks)
{
    static int resident = 0;
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_node<T, STAGE, DMI, OWN>, kTX * kTY<T>, 0);
        resident = (sms > 0 && per_sm > 0) ? sms * per_sm : 4 * 152;
    }
    NodeGrid ng{};
    ng.bxn = div_up(g.nn1, kTX);
    const int tiles = ng.bxn * div_up(g.nn2, kTY<T>);
    const int tail = tiles % resident;
    ng.full = tiles - tail;
    int chunks = tail > 0 ? resident / tail : 1;
    chunks = chunks < 1 ? 1 : (chunks > g.nn3 ? g.nn3 : chunks);
    ng.zc = div_up(g.nn3, chunks);
    ng.chunks = div_up(g.nn3, ng.zc);
    *blocks = ng.full + tail * ng.chunks;
    return ng;
}

template <typename T>
void launch_heff(const LocalParams<T> &p, const T *y, T *h_out, double t, cudaStream_t st)
{
    if (p.g.basis == 2) {
        k_node2d<T, false><<<dim3(div_up(p.g.nn1, 32), div_up(p.g.nn2, 8)), 256, 0, st>>>(p, y, h_out, nullptr,
                                                                                          StageArgs{}, t);
        return;
    }
    if (p.g.basis == 1) {
        k_node1d<T, false><<<p.g.nn1, kNode1dThreads, 0, st>>>(p, y, h_out, nullptr, StageArgs{}, t);
        return;
    }
    int nb;
    if (p.hdmi) {
        const NodeGrid ng = node_grid<T, false, true>(p.g, &nb);
        k_dmi<T><<<div_up(p.g.n_nodes, 256), 256, 0, st>>>(p, y, p.hdmi);
        k_node<T, false, true><<<nb, kTX * kTY<T>, 0, st>>>(p, y, h_out, nullptr, StageArgs{}, t, ng);
        return;
    }
    const NodeGrid ng = node_grid<T, false, false>(p.g, &nb);
    k_node<T, false><<<nb, kTX * kTY<T>, 0, st>>>(p, y, h_out, nullptr, StageArgs{}, t, ng);
}

template <typename T>
void launch_llg_stage(const LocalParams<T> &p, const T *y, T *k_out, T *y_next, const StageArgs &sa, cudaStream_t st)
{
    if (p.g.basis == 2) {
        k_node2d<T, true><<<dim3(div_up(p.g.nn1, 32), div_up(p.g.nn2, 8)), 256, 0, st>>>(p, y, k_out, y_next, sa,
                                                                                         0.0);
        return;
    }
    if (p.g.basis == 1) {
        k_node1d<T, true><<<p.g.nn1, kNode1dThreads, 0, st>>>(p, y, k_out, y_next, sa, 0.0);
        return;
    }
    int nb;
    if (p.hdmi) {
        const NodeGrid ng = node_grid<T, true, true>(p.g, &nb);
        k_dmi<T><<<div_up(p.g.n_nodes, 256), 256, 0, st>>>(p, y, p.hdmi);
        k_node<T, true, true><<<nb, kTX * kTY<T>, 0, st>>>(p, y, k_out, y_next, sa, 0.0, ng);
        return;
    }
    if constexpr (sizeof(T) == 4) {
        int n_earlier = 0;  // earlier slopes with non-zero coefficients in the next stage input
        for (int j = 0; j + 1 < sa.s && j < 7; ++j) n_earlier += sa.af[j] != 0.f;
        if (y_next && sa.mf && n_earlier >= 3 && n_earlier <= kOwnSlopes) {
            static bool carveout = false;  // six 32 KB blocks per SM: ask for the largest shared carveout
            if (!carveout) {
                cudaFuncSetAttribute((const void *)k_node<float, true, false, true>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
                carveout = true;
            }
            const NodeGrid ng = node_grid<T, true, false, true>(p.g, &nb);
            k_node<T, true, false, true><<<nb, kTX * kTY<T>, 0, st>>>(p, y, k_out, y_next, sa, 0.0, ng);
            return;
        }
    }
    const NodeGrid ng = node_grid<T, true, false>(p.g, &nb);
    k_node<T, true><<<nb, kTX * kTY<T>, 0, st>>>(p, y, k_out, y_next, sa, 0.0, ng);
}

// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_mass(Geom g, const double *__restrict__ Ms, double Ms0, double mu0V8, T *inv_mass,
                       unsigned long long *n_active)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= g.n_nodes) return;
    const int n1 = (int)(n % g.nn1);
    const long r = n / g.nn1;
    const int n2 = (int)(r % g.nn2);
    const int n3 = (int)(r / g.nn2);
    double s = 0.0;
    if (g.basis == 2) {
        // the 2D basis function of the node column is constant along z: the 4 in-plane cells of every
        // layer hold it, each with integral V/4 (twice the 3D corner share)
        for (int i = 0; i < 4; ++i) {
            const int c1 = n1 - ((i >> 1) & 1), c2 = n2 - (i & 1);
            if (c1 < 0 || c1 >= g.N1 || c2 < 0 || c2 >= g.N2) continue;
            for (int c3 = 0; c3 < g.N3; ++c3) s += 2.0 * (Ms ? Ms[((long)c3 * g.N2 + c2) * g.N1 + c1] : Ms0);
        }
    } else if (g.basis == 1) {
        // the 1D basis function is constant over the cross-section: every cell of the two slabs beside
        // the node holds it, each with integral V/2 (four times the 3D corner share)
        for (int c1 = n1 - 1; c1 <= n1; ++c1) {
            if (c1 < 0 || c1 >= g.N1) continue;
            for (long j = 0; j < (long)g.N2 * g.N3; ++j) s += 4.0 * (Ms ? Ms[j * g.N1 + c1] : Ms0);
        }
    } else {
        for (int i = 0; i < 8; ++i) {
            int c1 = n1 - ((i >> 2) & 1), c2 = n2 - ((i >> 1) & 1), c3 = n3 - (i & 1);
            if (c1 >= 0 && c1 < g.N1 && c2 >= 0 && c2 < g.N2 && c3 >= 0 && c3 < g.N3)
                s += Ms ? Ms[((long)c3 * g.N2 + c2) * g.N1 + c1] : Ms0;
        }
    }
    double mass = mu0V8 * s;
    inv_mass[n] = mass > 0.0 ? (T)(1.0 / mass) : T(0);
    if (mass > 0.0) atomicAdd(n_active, 1ull);
}

template <typename T>
void launch_mass(const Geom &g, const double *Ms_d, double Ms0, double V, T *inv_mass, unsigned long long *n_active,
                 cudaStream_t st)
{
    k_mass<T><<<div_up(g.n_nodes, 256), 256, 0, st>>>(g, Ms_d, Ms0, kMu0 * V / 8.0, inv_mass, n_active);
}

template void launch_heff<float>(const LocalParams<float> &, const float *, float *, double, cudaStream_t);
template void launch_heff<double>(const LocalParams<double> &, const double *, double *, double, cudaStream_t);
template void launch_llg_stage<float>(const LocalParams<float> &, const float *, float *, float *, const StageArgs &,
                                      cudaStream_t);
template void launch_llg_stage<double>(const LocalParams<double> &, const double *, double *, double *,
                                       const StageArgs &, cudaStream_t);
template void launch_mass<float>(const Geom &, const double *, double, double, float *, unsigned long long *,
                                 cudaStream_t);
template void launch_mass<double>(const Geom &, const double *, double, double, double *, unsigned long long *,
                                  cudaStream_t);

}  // namespace nm
