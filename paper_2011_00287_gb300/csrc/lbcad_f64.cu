// FP64 instantiation: populations stored unshifted (the plain FP64 path).
#include "lbcad_fused.cuh"
template struct lbcad::Launch<double, false>;
template struct lbcad::LaunchFused<double, false>;
