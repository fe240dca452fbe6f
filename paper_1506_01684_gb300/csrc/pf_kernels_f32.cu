// FP32 instantiation of the phase-field kernels (fused multiply-add allowed).
#define PF_FLOAT_UNIT 1
#include "pf_kernels.cuh"
namespace pf {
PF_INSTANTIATE(float)
}
