// FP64 instances of the demag passes (templates in demag_impl.cuh).
#include "demag_impl.cuh"

namespace nm {

void demag_init_attributes_f64() { init_attributes_t<double>(); }

template DemagPlan demag_plan<double>(const Geom &);
template void demag_forward<double>(const Geom &, const DemagBufs<double> &, const double *, double *, cudaStream_t);
template void demag_cells<double>(const Geom &, const DemagBufs<double> &, const double *, double *, cudaStream_t);
template int demag_encode_ymap<double>(const Geom &, void *, CUtensorMap *);

}  // namespace nm
