// Reverse-mode (adjoint) kernels, FP32 instantiation.
#include "lbcad_adjoint.cuh"
template struct lbcad::LaunchAdj<float, true>;
