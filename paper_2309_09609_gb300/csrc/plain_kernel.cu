// plain_kernel.cu -- the baseline of libswgb: Algorithm 1 of arxiv 2309.09609
// verbatim in int32 (E, F, H and S per cell, 5 additions/subtractions and 6
// maxima), one thread per subject of a 64-subject group, PT query rows per
// thread with an int32 profile in shared memory, one launch per query, and no
// separate path for long subjects.
#include "device_common.cuh"

namespace swgb {

constexpr int PT = 8;  // query rows per thread
constexpr int NEG = -(1 << 28);

__global__ void __launch_bounds__(GROUP)
plain_kernel(DbView db, const SearchParams* __restrict__ P, int q, int2* border,
             const int64_t* __restrict__ border_off) {
  __shared__ int8_t sm[NCODES * NCODES];
  __shared__ int prof[NCODES][PT];
  load_matrix(sm, P);
  const int k = threadIdx.x;  // subject slot in the group
  const int m = P->qlen[q];
  const uint8_t* __restrict__ qr = P->qres + P->qoff[q];
  const int go = P->go, ge = P->ge;
  int2* bd = border + border_off[blockIdx.x] + k;
  __syncthreads();
  for (int g = blockIdx.x; g < db.groups; g += gridDim.x) {
    const int L = db.glen[g];
    const uint2* __restrict__ res = (const uint2*)(db.inter + db.goff[g]) + k;
    const int nstrips = L > 0 ? (m + PT - 1) / PT : 0;
    int S = 0;
    for (int s = 0; s < nstrips; s++) {
      __syncthreads();
      for (int i = threadIdx.x; i < NCODES * PT; i += blockDim.x) {
        const int c = i / PT, r = i % PT, row = s * PT + r;
        prof[c][r] = row < m ? (int)sm[(int)qr[row] * NCODES + c] : PAD_SCORE;
      }
      __syncthreads();
      int Hl[PT], El[PT];
#pragma unroll
      for (int r = 0; r < PT; r++) {
        Hl[r] = 0;
        El[r] = NEG;
      }
      int hul = 0;
      const bool last = (s == nstrips - 1);
      for (int c = 0; c < L / CHUNK; c++) {
        const uint2 rr = res[c * GROUP];
#pragma unroll
        for (int jj = 0; jj < CHUNK; jj++) {
          const int cj = ((jj < 4 ? rr.x : rr.y) >> (8 * (jj & 3))) & 0xff;
          int hu = 0, fu = NEG;  // H and F of the row above the strip
          if (s > 0) {
            const int2 v = bd[(c * CHUNK + jj) * GROUP];
            hu = v.x;
            fu = v.y;
          }
          int hd = hul;
          hul = hu;
#pragma unroll
          for (int r = 0; r < PT; r++) {
            // Algorithm 1: E, F, H, S
            const int e = max(El[r] - ge, Hl[r] - go);
            const int f = max(fu - ge, hu - go);
            int h = hd + prof[cj][r];
            h = max(h, e);
            h = max(h, f);
            h = max(h, 0);
            S = max(h, S);
            hd = Hl[r];
            Hl[r] = h;
            El[r] = e;
            hu = h;
            fu = f;
          }
          if (!last) bd[(c * CHUNK + jj) * GROUP] = make_int2(hu, fu);
        }
      }
    }
    const int orig = db.perm[g * GROUP + k];
    if (orig >= 0) P->scores[(int64_t)q * db.n + orig] = S;
  }
}

int plain_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, plain_kernel, GROUP, 0) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_plain(int blocks, const DbView& db, const SearchParams* params, int query,
                         int2* border, const int64_t* border_off, cudaStream_t stream) {
  cudaGetLastError();  // a stale error must not be read as this launch's
  plain_kernel<<<blocks, GROUP, 0, stream>>>(db, params, query, border, border_off);
  return cudaGetLastError();
}

}  // namespace swgb
