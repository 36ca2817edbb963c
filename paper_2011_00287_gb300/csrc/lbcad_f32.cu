// FP32 instantiation: populations stored shifted by their rest weights, f_i - w_i rho0.
#include "lbcad_fused.cuh"
template struct lbcad::Launch<float, true>;
template struct lbcad::LaunchFused<float, true>;
