// FP64 instantiation of the solver kernels (depth form).  Compiled with
// -fmad=false: no multiply-add contraction, so each expression rounds as
// written and the FP64 path can be compared with the FP64 CPU oracle to
// round-off.
#include "mwdg_kernels.cuh"

template struct mwdg::Launch<double>;
