// ts_all.cu -- libts.so is compiled as one CUDA translation unit, so every
// kernel (template instantiations included) is launched from the unit that
// defines it.
#include "ts_neighbor.cu"
#include "ts_relist_small.cu"
#include "ts_pair.cu"
#include "ts_md.cu"
#include "ts_run.cu"
#include "ts_api.cu"
#include "ts_fire.cu"
#include "ts_adjoint.cu"
#include "ts_inflight.cu"
#include "ts_tune.cu"
#include "ts_noalloc.cu"
