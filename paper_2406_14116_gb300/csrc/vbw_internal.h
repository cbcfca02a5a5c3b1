// Host-side definitions shared by the translation units of libvbw (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "vbw.h"
#include "vbw_common.cuh"

struct vbw_plan_s {
    int N = 0, O = 0, M = 0, LV = 0, prec = 0;
    int device = 0, sms = 0;
    std::vector<double> V;
    float2* d_tw = nullptr;
    float* d_V = nullptr;
    int* d_status = nullptr;         // device status word of this plan's launches (bit flags)
    unsigned char* d_tc = nullptr;   // tensor-core precisions: DFT-matrix pieces and twiddles
};

// vbw_api.cu
vbw_status fail(vbw_status st, const char* fmt, ...);   // sets vbw_last_error() text
vbw_status ok();
vbw_status check_band(const vbw_plan_s* p, int band);
bool misaligned(const void* p);
void fill_plan_args(vbw::OlsArgs& a, const vbw_plan_s* p);
cudaError_t launch_plan(const vbw_plan_s* p, const vbw::OlsArgs& a, cudaStream_t st, int max_ctas = 0);
// Blocks per work tile: one warp-tile of the FP32 kernel, or the 8-block tile of the tensor-core one.
int tile_blocks(const vbw_plan_s* p);
