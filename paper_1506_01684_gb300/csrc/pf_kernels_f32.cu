// FP32 instantiation of the phase-field kernels (fused multiply-add allowed).
#include "pf_kernels.cuh"
namespace pf {
PF_INSTANTIATE(float)
}
