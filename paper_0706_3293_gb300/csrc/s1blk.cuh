// s1blk.cuh -- host entry points of the s = 1 block-structured products (s1blk.cu); the
// plan and the device bodies are in s1_sweep.cuh.
#pragma once

#include "hm_internal.cuh"
#include "s1_sweep.cuh"

namespace hm {

static_assert(S1_MAXK == S1_KMAX && S1_LWOFF >= 2 * S1_KMAX + 2, "s = 1 split limits disagree");

// plan of the s = 1 block path for these bonds; 1 when it does not apply (the caller runs
// the general row kernel), < 0 on error.  Builds the basis's tables on first use.
int s1_plan(hm_basis *b, const BondParams &bp, S1Plan *P);
// y = H x, FP32, one vector
int s1_matvec(const S1Plan &P, const float *x, float *y, cudaStream_t st);
// Lanczos product, FP32: q_prev <- sigma H q - gamma q_prev; part[block] = (sigma q . u)
int s1_lz32(const S1Plan &P, const float *qc, float *qp, const LzScalars *S, double *part, cudaStream_t st);
// Lanczos product, FP64 (kernel specialised to the bonds; 1 when it cannot be compiled):
// Y <- H q as binary64 bit patterns from the fixed-point copy Xc of q (exponent
// S->emax[pc]); part[block] = (q . y)
int s1_lz64(const S1Plan &P, const long long *Xc, unsigned long long *Y, const LzScalars *S, int pc, double *part,
            cudaStream_t st);
// whether the specialised kernel of mode m (0 s1_matvec, 1 s1_lz32, 2 s1_lz64) serves
// plan P (compiles it on first use; modes 0 and 1 have a generic fallback)
bool s1_jit_ready(const S1Plan &P, int mode);
// name of the kernel s1_matvec (mode 0), s1_lz32 (1) or s1_lz64 (2) launches for plan P
const char *s1_kernel_name(const S1Plan &P, int mode);
// number of blocks of a basis's s = 1 path with K = min(10, N - 2) (0 when it does not apply)
uint64_t s1_block_count(const hm_basis *b);

// kernels of plan P specialised to its bonds (jit.cu): mode 0 y = H x FP32, 1 Lanczos
// FP32, 2 Lanczos FP64; 0 and the handle, or 1 when NVRTC cannot serve
int jit_s1_kernel(const S1Plan &P, int mode, const void **kern);

}  // namespace hm
