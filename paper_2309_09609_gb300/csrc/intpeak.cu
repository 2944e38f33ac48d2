// intpeak.cu -- integer-pipe throughput microbenchmark.
//
// The paper's peak model (Section III-B, Eq. 4-5) multiplies clock rate,
// per-lane instruction throughput, lanes and cores, then divides by the
// instructions one cell update needs.  Its throughput column comes from
// vendor tables; for sm_103a there is no such table for the 16x2 SIMD and
// DPX instructions this library uses, so it is measured here: many warps run
// independent chains of one instruction kind; the lane-operations completed
// per SM clock give the per-SM throughput, and SM count x clock x that rate is
// the roofline denominator for the alignment kernels.
//
// Each "op" below is one lane instruction of a given kind (or a fixed mix).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include "swgb_internal.h"

namespace swgb {

enum IntOp {
  OP_IADD = 0,         // int32 add
  OP_IMAX = 1,         // int32 max
  OP_VIADDMAX_S32 = 2, // DPX max(a + b, c), int32
  OP_VIADDMAX_S16X2 = 3,
  OP_VIADDMAX_S16X2_RELU = 4,
  OP_VIMAX3_S16X2 = 5,
  OP_VMAXS2 = 6,       // SIMD-video signed 16x2 max
  OP_VSUB2 = 7,        // 16x2 wrapping subtract
  OP_VADDSS2 = 8,      // 16x2 saturating add
  OP_PRMT = 9,         // byte permute
  OP_CELL_S16X2 = 10,  // one packed cell-pair update (6 ops, see below)
  OP_CELL_S16X2_PRMT = 11, // the same plus one PRMT (7 ops)
  OP_CELL_I32 = 12,    // Algorithm 1 style int32 cell (10 ops after sharing H-Go)
  OP_IMAD = 13,        // int32 multiply-add with a run-time multiplier (FMA pipe)
  OP_CELL_BIASED = 14, // the packed cell pair of the search kernel: prmt, vimax3,
                       // viaddmax, imad (H'-Go), viaddmax x2 (6 ops, one on the FMA pipe)
  // 8-bit SIMD (four cells per word), for the int8x4 question
  OP_VADD4 = 15,       // 8x4 wrapping add
  OP_VMAXU4 = 16,      // 8x4 unsigned max
  OP_VMAXS4 = 17,      // 8x4 signed max
  OP_VADDUS4 = 18,     // 8x4 unsigned saturating add
  OP_VSUBUS4 = 19,     // 8x4 unsigned saturating subtract
  OP_CELL_U8X4 = 20,   // an unsigned biased 8x4 cell update (four cells): addus, subus,
                       // maxu x2 (E, F), subus (H - Go), subus x2 (E, F - Ge), maxu x2,
                       // maxu (S) -- 10 ops
  OP_COUNT = 21
};

__host__ __device__ inline int intpeak_ops_per_step(int op) {
  switch (op) {
    case OP_CELL_S16X2: return 6;
    case OP_CELL_S16X2_PRMT: return 7;
    case OP_CELL_I32: return 10;
    case OP_CELL_BIASED: return 6;
    case OP_CELL_U8X4: return 10;
    default: return 1;
  }
}

#define CHAINS 8

template <int OP>
__device__ __forceinline__ void step(uint32_t (&a)[CHAINS], uint32_t c0, uint32_t c1,
                                     uint32_t one) {
#pragma unroll
  for (int i = 0; i < CHAINS; i++) {
    uint32_t x = a[i], y = a[(i + 1) % CHAINS];
    uint32_t r;
    if (OP == OP_IADD) r = x + (y ^ c0);
    else if (OP == OP_IMAX) r = (uint32_t)max((int)x, (int)(y + c0));
    else if (OP == OP_VIADDMAX_S32) r = (uint32_t)__viaddmax_s32((int)x, (int)c0, (int)y);
    else if (OP == OP_VIADDMAX_S16X2) r = __viaddmax_s16x2(x, c0, y);
    else if (OP == OP_VIADDMAX_S16X2_RELU) r = __viaddmax_s16x2_relu(x, c0, y);
    else if (OP == OP_VIMAX3_S16X2) r = __vimax3_s16x2(x, y, c1);
    else if (OP == OP_VMAXS2) r = __vmaxs2(x, y);
    else if (OP == OP_VSUB2) r = __vsub2(x, y);
    else if (OP == OP_VADDSS2) r = __vaddss2(x, y);
    else if (OP == OP_PRMT) r = __byte_perm(x, y, 0xC480 + (i & 3) * 0x1111);
    else if (OP == OP_VADD4) r = __vadd4(x, y);
    else if (OP == OP_VMAXU4) r = __vmaxu4(x, y);
    else if (OP == OP_VMAXS4) r = __vmaxs4(x, y);
    else if (OP == OP_VADDUS4) r = __vaddus4(x, y);
    else if (OP == OP_VSUBUS4) r = __vsubus4(x, y);
    else if (OP == OP_CELL_U8X4) {
      // x: H diag / F, y: biased profile word / E; c0 = Go (x4), c1 = Ge (x4).
      // Unsigned saturation at 0 gives the zero term of Eq. 1 for free.
      uint32_t h = __vsubus4(__vaddus4(x, y), c0 ^ c1);  // H = hd + (w + bias) - bias
      h = __vmaxu4(h, __vmaxu4(x, y));                    // max(., E, F)
      const uint32_t t = __vsubus4(h, c0);                 // H - Go
      const uint32_t e = __vmaxu4(__vsubus4(y, c1), t);    // Eq. 2
      const uint32_t f = __vmaxu4(__vsubus4(x, c1), t);    // Eq. 3
      r = __vmaxu4(e, f) ^ h;                              // S-like fold
    }
    else if (OP == OP_IMAD) {
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(c1), "r"(y));
    } else if (OP == OP_CELL_BIASED) {
      // x: H' diag / F', y: profile source / E'; c0 = Go (both halves), c1 = -Ge
      uint32_t p, t;
      asm("prmt.b32 %0, %1, %2, 0xC480;" : "=r"(p) : "r"(y), "r"(x));
      uint32_t h = __viaddmax_s16x2(x, p, __vimax3_s16x2(y, x, c0));
      asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(t) : "r"(h), "r"(one), "r"(c1));
      uint32_t e = __viaddmax_s16x2(y, c1, t);
      uint32_t f = __viaddmax_s16x2(x, c1, t);
      r = e ^ f;
    }
    else if (OP == OP_CELL_S16X2 || OP == OP_CELL_S16X2_PRMT) {
      // x plays H-diag, y the profile word / E, c0 = -Go packed, c1 = -Ge packed
      uint32_t p = y;
      if (OP == OP_CELL_S16X2_PRMT) p = __byte_perm(y, x, 0xC480);
      uint32_t ef = __vmaxs2(y, x);
      uint32_t h = __viaddmax_s16x2_relu(x, p, ef);
      uint32_t t = __vsub2(h, c0);
      uint32_t e = __viaddmax_s16x2(y, c1, t);
      uint32_t f = __viaddmax_s16x2(x, c1, t);
      r = __vmaxs2(e, f);
    } else {  // OP_CELL_I32: e/f/h/max in plain int32
      int xi = (int)x, yi = (int)y, go = (int)c0, ge = (int)c1;
      int e = max(yi - ge, xi - go);
      int f = max(xi - ge, yi - go);
      int h = max(max(xi + (yi & 15), e), max(f, 0));
      int s = max(h, yi);
      int t = h - go;
      r = (uint32_t)(max(e - ge, t) ^ s);
    }
    a[i] = r;
  }
}

template <int OP>
__global__ void intpeak_kernel(int iters, uint32_t seed, uint32_t* sink, long long* cycles) {
  uint32_t a[CHAINS];
#pragma unroll
  for (int i = 0; i < CHAINS; i++) a[i] = seed * (threadIdx.x + 1) + i * 0x9E3779B9u;
  uint32_t c0 = seed ^ 0x00050005u, c1 = seed ^ 0x00020002u;
  const uint32_t one = (seed >> 31) | 1u;  // 1, not known at compile time
  long long t0 = clock64();
  for (int it = 0; it < iters; it++) {
    step<OP>(a, c0, c1, one);
  }
  long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < CHAINS; i++) acc ^= a[i];
  // the write is data dependent, so no chain can be dropped
  if (acc == seed) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

typedef void (*IntpeakKernel)(int, uint32_t, uint32_t*, long long*);

static IntpeakKernel intpeak_pick(int op) {
  switch (op) {
    case OP_IADD: return intpeak_kernel<OP_IADD>;
    case OP_IMAX: return intpeak_kernel<OP_IMAX>;
    case OP_VIADDMAX_S32: return intpeak_kernel<OP_VIADDMAX_S32>;
    case OP_VIADDMAX_S16X2: return intpeak_kernel<OP_VIADDMAX_S16X2>;
    case OP_VIADDMAX_S16X2_RELU: return intpeak_kernel<OP_VIADDMAX_S16X2_RELU>;
    case OP_VIMAX3_S16X2: return intpeak_kernel<OP_VIMAX3_S16X2>;
    case OP_VMAXS2: return intpeak_kernel<OP_VMAXS2>;
    case OP_VSUB2: return intpeak_kernel<OP_VSUB2>;
    case OP_VADDSS2: return intpeak_kernel<OP_VADDSS2>;
    case OP_PRMT: return intpeak_kernel<OP_PRMT>;
    case OP_CELL_S16X2: return intpeak_kernel<OP_CELL_S16X2>;
    case OP_CELL_S16X2_PRMT: return intpeak_kernel<OP_CELL_S16X2_PRMT>;
    case OP_CELL_I32: return intpeak_kernel<OP_CELL_I32>;
    case OP_IMAD: return intpeak_kernel<OP_IMAD>;
    case OP_CELL_BIASED: return intpeak_kernel<OP_CELL_BIASED>;
    case OP_VADD4: return intpeak_kernel<OP_VADD4>;
    case OP_VMAXU4: return intpeak_kernel<OP_VMAXU4>;
    case OP_VMAXS4: return intpeak_kernel<OP_VMAXS4>;
    case OP_VADDUS4: return intpeak_kernel<OP_VADDUS4>;
    case OP_VSUBUS4: return intpeak_kernel<OP_VSUBUS4>;
    case OP_CELL_U8X4: return intpeak_kernel<OP_CELL_U8X4>;
    default: return nullptr;
  }
}

// Runs one measurement.  Fills lane-ops per SM clock, the SM clock (MHz)
// derived from clock64 cycles over CUDA-event time, and the elapsed seconds.
int intpeak_run(int op, int blocks_per_sm, int threads, int iters, double* lane_ops_per_clk_sm,
                double* clock_mhz, double* seconds) {
  IntpeakKernel k = intpeak_pick(op);
  if (!k || blocks_per_sm < 1 || threads < 32 || threads > 1024 || iters < 1) return SW_EINVAL;
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int grid = sms * blocks_per_sm;
  uint32_t* sink = nullptr;
  long long* cyc = nullptr;
  CUDA_TRY(cudaMalloc(&sink, sizeof(uint32_t) * (size_t)grid * threads));
  CUDA_TRY(cudaMalloc(&cyc, sizeof(long long) * grid));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k<<<grid, threads>>>(iters / 8 + 1, 12345u, sink, cyc);  // warm-up
  cudaEventRecord(e0);
  k<<<grid, threads>>>(iters, 12345u, sink, cyc);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  long long* hc = new long long[grid];
  cudaMemcpy(hc, cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
  double maxc = 0;
  for (int i = 0; i < grid; i++) maxc = hc[i] > maxc ? (double)hc[i] : maxc;
  delete[] hc;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(cyc);
  if (err != cudaSuccess) return sw_set_cuda_error(err, "intpeak");
  double lane_ops = (double)grid * threads * (double)iters * CHAINS * intpeak_ops_per_step(op);
  double secs = ms * 1e-3;
  // blocks_per_sm blocks share an SM; the slowest block's cycle count bounds the SM
  *lane_ops_per_clk_sm = lane_ops / sms / maxc;
  *clock_mhz = maxc / secs / 1e6;
  *seconds = secs;
  return SW_OK;
}

}  // namespace swgb

#ifdef INTPEAK_MAIN
int main() {
  const char* names[] = {"iadd", "imax", "viaddmax_s32", "viaddmax_s16x2", "viaddmax_s16x2_relu",
                         "vimax3_s16x2", "vmaxs2", "vsub2", "vaddss2", "prmt", "cell_s16x2",
                         "cell_s16x2_prmt", "cell_i32", "imad", "cell_biased", "vadd4", "vmaxu4",
                         "vmaxs4", "vaddus4", "vsubus4", "cell_u8x4"};
  for (int op = 0; op < swgb::OP_COUNT; op++) {
    for (int bps : {4, 8}) {
      double r, mhz, s;
      int rc = swgb::intpeak_run(op, bps, 256, 20000, &r, &mhz, &s);
      printf("%-20s bps=%d rc=%d lane_ops/clk/SM=%.1f clock=%.0fMHz t=%.1fms\n", names[op], bps,
             rc, r, mhz, s * 1e3);
    }
  }
  return 0;
}
#endif
