// FP32 instances of the demag passes (templates in demag_impl.cuh).
#include "demag_impl.cuh"

namespace nm {

void demag_init_attributes_f64();

void demag_init_attributes()
{
    static bool done = false;
    if (done) return;
    init_attributes_t<float>();
    demag_init_attributes_f64();
    done = true;
}

template DemagPlan demag_plan<float>(const Geom &);
template void demag_forward<float>(const Geom &, const DemagBufs<float> &, const float *, float *, cudaStream_t);
template void demag_cells<float>(const Geom &, const DemagBufs<float> &, const float *, float *, cudaStream_t);
template int demag_encode_ymap<float>(const Geom &, void *, CUtensorMap *);

}  // namespace nm
