// Demag tensor set-up (FP64) and its spectrum in the layout the convolution passes read.
#pragma once
#include "demag.cuh"

namespace nm {

// Nk[comp][kz'][ky'][kx] (comp order xx yy zz xy xz yz, kz' < H3, ky' < H2, kx < Xp), scaled by
// -1/(P1 P2 P3) so that the inverse transform of Nk * M^ is the cell field directly.
template <typename T>
cudaError_t build_tensor_spectrum(const Geom &g, double a, double b, double c, const Cx<double> *tw64, T *Nk,
                                  cudaStream_t st);

// Real-space tensor octant out[comp][d3][d2][d1] for offsets d in [0,N1) x [0,N2) x [0,N3).
cudaError_t newell_octant(int N1, int N2, int N3, double a, double b, double c, double *out, cudaStream_t st);

}  // namespace nm
