// FP64 instantiation: populations stored unshifted (the plain FP64 path).
#include "lbcad_kernels.cuh"
template struct lbcad::Launch<double, false>;
