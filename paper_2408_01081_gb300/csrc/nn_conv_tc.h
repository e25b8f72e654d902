// Internal interface of the tcgen05 3x3 convolution (nn_conv_tc.cu), called by
// the convolution entry point of nn_kernels.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct ConvTcArgs {
    const float* x1;            // first input, C1 channels, [B][H][W][C1] (or [B][H/2][W/2][C1] with x1_half)
    const float* x2;            // second input (channels after x1), C2 channels, or null
    int C1, C2;                 // multiples of 32
    const uint16_t* w;          // BF16 weights [Cout][3][3][C1 + C2]
    const float* bias;          // [Cout] or null
    float* y1;                  // output channels [0, Co1)
    float* y2;                  // output channels [Co1, Cout), or null
    int Co1, Cout;              // Co1 a multiple of 16
    int B, H, W;                // powers of two
    int relu, beta, x1_half, act_bf16;
};

// Launches the tensor-core convolution when its tiling applies to these sizes and
// returns true; returns false (nothing launched) otherwise, and the caller uses
// another kernel.  `stages` = 0 picks the pipeline depth.
bool conv3_tc_launch(const ConvTcArgs& a, cudaStream_t s, int stages);

// Reads and clears the flag that a bounded wait inside the kernel ran out
// (the output of that launch is invalid); synchronises `s`.
bool conv3_tc_take_timeout(cudaStream_t s);
