// FP64 instantiation of the phase-field kernels.  This unit is compiled without fused
// multiply-add contraction (-fmad=false) so that its rounding follows the written
// expressions, like the FP64 CPU oracle it is checked against.
#include "pf_kernels.cuh"
namespace pf {
PF_INSTANTIATE(double)
}
