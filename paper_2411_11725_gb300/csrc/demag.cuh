// Demagnetising field by zero-padded FFT convolution on the cell grid with node->cell and
// cell->node averaging (section "Demagnetization Field" of the paper).  The padded transform is
// never materialised: every pass reads only the non-zero part of its input and writes only the part
// of its output that later passes use.
#pragma once
#include <cuda.h>  // CUtensorMap (descriptor type only; the encoder is reached through the runtime)

#include "nm_common.cuh"

namespace nm {

struct Geom {
    int N1, N2, N3;            // cells
    int nn1, nn2, nn3;         // nodes = cells + 1 (nn3 = 1 with the 2D basis, nn2 = nn3 = 1 with the 1D)
    int basis;                 // 3: trilinear nodal basis; 2: 2D nodal basis, constant along z over all N3
                               // cell layers; 1: 1D nodal basis, constant along y and z over the whole
                               // cross-section (section "Low-Dimensional Geometries")
    int zsn;                   // node offset between the z corners of a cell: nn1 nn2 (3D) or 0 (2D, 1D)
    long n_nodes, n_cells;
    long ns;                   // component stride of nodal SoA arrays
    long cs;                   // component stride of cell SoA arrays
    int P1, P2, P3;            // padded FFT lengths (1 when N_k == 1)
    int Q, lgQ, lgP2, lgP3;    // Q = P1/2 (complex length of the x transform), 0 when P1 == 1
    int X, Xp;                 // X = P1/2 + 1 half-spectrum length, Xp = X padded for grouping
    int H2, H3;                // tensor octant lengths P2/2+1, P3/2+1
    int twlg;                  // log2 of the twiddle table length
    long s_comp;               // component stride of the spectrum buffer = N3 * P2 * Xp
    long t_comp;               // component stride of the tensor spectrum = H3 * H2 * Xp
    FastDiv n2f;               // division by N2 (cell row -> (y, z))
    int ysn;                   // node offset between the y corners of a cell: nn1 (3D, 2D) or 0 (1D)
};

template <typename T>
struct DemagBufs {
    Cx<T> *S;                  // spectra [3][N3][P2][Xp]
    const T *Nk;               // tensor spectrum [6][H3][H2][Xp], already scaled by -1/(P1 P2 P3)
    const Cx<T> *tw;           // twiddle table e^{-2 pi i k / 2^twlg}
    const T *Ms;               // cell Ms map (SoA, n_cells) or NULL for uniform
    T Ms0;
    const StepCtl *ctl;        // when set, passes do nothing once ctl->done (finished integrations)
    Marker mark;               // profiling hook
    // TMA descriptor of a y-pass tile over S, all P2 rows (the inverse pass's load and the forward pass's
    // store; host copy, passed to the kernels by value; built once per mesh by demag_encode_ymap)
    const CUtensorMap *ymap = nullptr;
    int *wait_err = nullptr;   // device status word set to NM_ERR_TIMEOUT when a bounded wait runs out
};

// Launch shapes of the passes (lines per block bounded by the FFT engine's 16 values per thread).
struct DemagPlan {
    bool ok;  // the grid fits the engine's per-block budget in this precision
    int x_lpb, x_threads;      // forward x pass
    size_t x_smem;
    int xi_lpb, xi_threads;    // inverse x pass
    size_t xi_smem;
    int y_G, y_threads;
    size_t y_smem;
    int z_G, z_KY, z_threads;
    size_t z_smem;
    bool z_reg;                // FP32, P3 <= 64: the register z convolution (two threads per line)
    int yc_G, yc_threads;
    size_t yc_smem;
    size_t yi_smem;            // y passes with a TMA tile (alignment slack and barrier)
};
template <typename T>
DemagPlan demag_plan(const Geom &g);

// Demag of the nodal field y (SoA, real T): writes (Ms_c H_c) per cell into MsH (3 x cs).
template <typename T>
void demag_forward(const Geom &g, const DemagBufs<T> &b, const T *y, T *MsH, cudaStream_t st);

// Same pipeline with an explicit cell input: M (3 x cs, already Ms-weighted cell magnetisation)
// replaces the node->cell averaging; output H (3 x cs) without the Ms factor.  Used by the adjoint.
template <typename T>
void demag_cells(const Geom &g, const DemagBufs<T> &b, const T *M, T *H, cudaStream_t st);

// TMA descriptor of a y-pass tile over the spectrum buffer S (host work only; no device access).
// Returns 0, or a non-zero code when the driver's encoder is unavailable or refuses the shape.
template <typename T>
int demag_encode_ymap(const Geom &g, void *S, CUtensorMap *map);

// Raise the dynamic shared-memory limit of every demag kernel once (outside any graph capture).
void demag_init_attributes();

}  // namespace nm
