// Tensor-core D_hat line sweeps of the FP32 precision form.
//
// A sweep along direction l is a batched small matrix product
//   C[line][i] = sum_a A[line][a] * Dhat[i][a],   A[line][a] = field at node(line, a),
// with one row per line of n nodes (lines of all fields and elements of the CTA
// flattened), K = n <= 8 and N = n <= 8.  Warps take 16-line tiles and issue
// mma.sync (m16n8k8 TF32 or m16n8k16 BF16) with FP32 accumulation; results are
// added into a shared per-node accumulator, one direction at a time.
//
// Split precision: TF32 keeps 11 significant bits and BF16 8, so each operand
// is split into three terms x1 + x2 + x3 of the narrow type (33 resp. 24
// bits, i.e. FP32-equivalent), and the six products of total order <= 2
// (A1B1, A1B2, A2B1, A1B3, A2B2, A3B1) are formed and accumulated in FP32,
// smallest first.  TF32 (m16n8k8) issues them as six mma; BF16 (m16n8k16)
// packs them pairwise into the K = 16 dimension:
// [A1|A3]x[B3;B1], [A1|A2]x[B2;B1], [A1|A2]x[B1;B2].
#pragma once
#include <cuda_bf16.h>

#include "dg_common.cuh"

namespace flexi {

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// pack (lo = x0, hi = x1) as bf16x2
__device__ __forceinline__ uint32_t pack_bf16(float x0, float x1) {
  __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void split3_tf32(float x, uint32_t& x1, uint32_t& x2, uint32_t& x3) {
  x1 = to_tf32(x);
  const float r1 = x - __uint_as_float(x1);
  x2 = to_tf32(r1);
  x3 = to_tf32(r1 - __uint_as_float(x2));
}

__device__ __forceinline__ void split3_bf16(float x, float& x1, float& x2, float& x3) {
  x1 = __bfloat162float(__float2bfloat16_rn(x));
  const float r1 = x - x1;
  x2 = __bfloat162float(__float2bfloat16_rn(r1));
  x3 = __bfloat162float(__float2bfloat16_rn(r1 - x2));
}

// B fragments of Dhat^T (B[a][i] = Dhat[i][a] = DhatT[a*n+i]) held per lane
template <int SW>
struct BFrag {
  uint32_t r[6];
};

template <int n, int SW>
__device__ __forceinline__ BFrag<SW> make_bfrag(const float* sD, int lane) {
  const int gid = lane >> 2, tig = lane & 3;
  BFrag<SW> f;
  auto B = [&](int a, int i) -> float { return (a < n && i < n) ? sD[a * n + i] : 0.f; };
  if (SW == 1) {
    // r[2t], r[2t+1]: term t of the rows (tig, tig + 4) at column gid
    split3_tf32(B(tig, gid), f.r[0], f.r[2], f.r[4]);
    split3_tf32(B(tig + 4, gid), f.r[1], f.r[3], f.r[5]);
  } else {
    float p0[3], p1[3];  // rows a = 2tig, 2tig+1 at column gid, three split terms
    split3_bf16(B(2 * tig, gid), p0[0], p0[1], p0[2]);
    split3_bf16(B(2 * tig + 1, gid), p1[0], p1[1], p1[2]);
    // K rows 0..7 hold the first factor's term, rows 8..15 the second's
    f.r[0] = pack_bf16(p0[0], p1[0]);  // B1
    f.r[1] = pack_bf16(p0[1], p1[1]);  // B2
    f.r[2] = pack_bf16(p0[2], p1[2]);  // B3
    f.r[3] = f.r[4] = f.r[5] = 0u;
  }
  return f;
}

// Accumulate sOut[el][v][node] (+)= sum over the 3 directions of the Dhat sweep of
// the 15 staged fields buf[el][l*5+v][node].  Block-wide; ends with __syncthreads.
template <int n, int NE, int SW>
__device__ __forceinline__ void tc_sweep3(const float* __restrict__ buf, float* __restrict__ sOut,
                                          const BFrag<SW>& bf, int tid, int T) {
  constexpr int n2 = n * n, n3p = Cfg<n>::n3p, P = Cfg<n>::P;
  constexpr int L = NE * NV * n2;  // lines per direction
  constexpr int tiles = (L + 15) / 16;
  const int warp = tid >> 5, lane = tid & 31;
  const int nwarps = T >> 5;  // only full warps issue mma
  const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    if (warp < nwarps) {
      for (int tile = warp; tile < tiles; tile += nwarps) {
        // the two rows (lines) this lane touches: gid and gid + 8
        int base[2], fld[2];
        bool ok[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int g = tile * 16 + gid + 8 * h;
          ok[h] = g < L;
          const int gg = ok[h] ? g : 0;
          const int el = gg / (NV * n2);
          const int rem = gg - el * NV * n2;
          const int v = rem / n2, line = rem - v * n2;
          fld[h] = (el * 15 + l * NV + v) * n3p;
          base[h] = l == 0 ? P * line : (l == 1 ? (line % n) + P * n * (line / n) : (line % n) + P * (line / n));
        }
        const int stride = l == 0 ? 1 : (l == 1 ? P : P * n);
        auto Aval = [&](int h, int a) -> float {
          return (ok[h] && a < n) ? buf[fld[h] + base[h] + stride * a] : 0.f;
        };
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        if (SW == 1) {
          uint32_t a[3][4];  // a[term][reg]: regs (row gid, col tig), (gid+8, tig), (gid, tig+4), (gid+8, tig+4)
          split3_tf32(Aval(0, tig), a[0][0], a[1][0], a[2][0]);
          split3_tf32(Aval(1, tig), a[0][1], a[1][1], a[2][1]);
          split3_tf32(Aval(0, tig + 4), a[0][2], a[1][2], a[2][2]);
          split3_tf32(Aval(1, tig + 4), a[0][3], a[1][3], a[2][3]);
          const uint32_t b1[2] = {bf.r[0], bf.r[1]}, b2[2] = {bf.r[2], bf.r[3]}, b3[2] = {bf.r[4], bf.r[5]};
          mma_tf32(c, a[2], b1);  // A3 B1
          mma_tf32(c, a[1], b2);  // A2 B2
          mma_tf32(c, a[0], b3);  // A1 B3
          mma_tf32(c, a[1], b1);  // A2 B1
          mma_tf32(c, a[0], b2);  // A1 B2
          mma_tf32(c, a[0], b1);  // A1 B1
        } else {
          float s00[3], s01[3], s10[3], s11[3];  // rows gid / gid+8, cols 2tig / 2tig+1
          split3_bf16(Aval(0, 2 * tig), s00[0], s00[1], s00[2]);
          split3_bf16(Aval(0, 2 * tig + 1), s01[0], s01[1], s01[2]);
          split3_bf16(Aval(1, 2 * tig), s10[0], s10[1], s10[2]);
          split3_bf16(Aval(1, 2 * tig + 1), s11[0], s11[1], s11[2]);
          auto afrag = [&](int p, int q, uint32_t a[4]) {
            a[0] = pack_bf16(s00[p], s01[p]);
            a[1] = pack_bf16(s10[p], s11[p]);
            a[2] = pack_bf16(s00[q], s01[q]);
            a[3] = pack_bf16(s10[q], s11[q]);
          };
          uint32_t a[4];
          const uint32_t b31[2] = {bf.r[2], bf.r[0]};
          afrag(0, 2, a);
          mma_bf16(c, a, b31);  // A1 B3 + A3 B1
          const uint32_t b21[2] = {bf.r[1], bf.r[0]};
          afrag(0, 1, a);
          mma_bf16(c, a, b21);  // A1 B2 + A2 B1
          const uint32_t b12[2] = {bf.r[0], bf.r[1]};
          mma_bf16(c, a, b12);  // A1 B1 + A2 B2
        }
        // scatter C[row][i] to the node accumulator
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!ok[h]) continue;
          const int g = tile * 16 + gid + 8 * h;
          const int el = g / (NV * n2);
          const int rem = g - el * NV * n2;
          const int v = rem / n2;
          float* out = sOut + (el * NV + v) * n3p + base[h];
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int i = 2 * tig + cc;
            if (i < n) {
              float* dst = out + stride * i;
              *dst = (l == 0 ? 0.f : *dst) + c[2 * h + cc];
            }
          }
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace flexi
