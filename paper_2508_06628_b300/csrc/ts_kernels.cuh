// ts_kernels.cuh -- libts.so is one CUDA translation unit (ts_all.cu): each
// kernel file is included before the host code that launches its kernels,
// so kernels need no forward declarations and template kernels are
// instantiated at their launch sites, after their definitions.
#pragma once
#include "ts_internal.cuh"
