// FP32 instantiation of the solver kernels (free-surface form eta = h + z;
// time, volume sums and the detail-threshold comparison stay FP64).
#include "mwdg_kernels.cuh"

template struct mwdg::Launch<float>;
