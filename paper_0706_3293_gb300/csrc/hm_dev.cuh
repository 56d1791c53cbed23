// hm_dev.cuh -- device definitions shared by the nvcc build and the kernels specialised
// at run time (jit.cu); compiles under nvcc and NVRTC alike (no host headers there).
#pragma once

#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#ifndef INT_MIN
#define INT_MIN (-2147483647 - 1)
#endif
#else
#include <stdint.h>
#include <stddef.h>
#include <climits>
#endif

namespace hm {

// device state of a Lanczos run (see lanczos.cu)
struct LzScalars {
    double sigma_cur;    // v_j = sigma_cur * q_cur (stored vectors are unnormalised)
    double sigma_prev;
    double beta_prev;
    double scale;        // max(|alpha_1..alpha_j|, beta_1..beta_{j-1})
    double nrm2;         // scratch for norms
    int j;               // steps done
    int done;
    int status;
    int mconv;           // e0_grad: Krylov length used
    int emax[2];         // largest exponent field of the vector held in buffer 0 / 1
    int emax_old;        // exponent of q_prev while its buffer receives w
    unsigned sched[2];   // block product: next block to hand out, CTAs finished (reset by the last)
};

// deterministic block reduction of doubles (fixed shuffle tree + fixed warp order)
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh /* >= NT/32 */) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < NT / 32; ++k) t += sh[k];
    return t;  // valid in thread 0
}

}  // namespace hm
