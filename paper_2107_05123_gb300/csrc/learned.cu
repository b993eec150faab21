// Learned coarse correction for the pressure-Poisson solve (an extension; the paper solves the
// Poisson system with PETSc's Krylov methods and has no learned component).
//
// * Grid transfer between the octree nodes and a uniform D^3 cell grid: trilinear interpolation
//   of cell-centred values at the nodes (P_g), its transpose (R = P_g^T, scatter with FP32
//   atomics) and the P_g-weighted cell mean of nodal fields.
// * A 4-level 3D convolutional U-Net with 16 channels. Activations are stored channel-last in
//   bfloat16 (one voxel = 16 channels = 32 bytes), so a 3x3x3 convolution is an implicit GEMM:
//   M = voxels, N = 16 output channels, K = 27 taps x 16 input channels. It runs on the tensor
//   cores with mma.sync m16n8k16 (bf16 x bf16 -> fp32): per CTA an 8x8x4 output tile, its
//   10x10x6 halo and all 27 weight taps staged in shared memory with a 48-byte voxel stride so
//   that every ldmatrix phase is free of bank conflicts. The transposed convolution of the
//   backward pass is the same kernel with flipped, transposed taps; the weight gradient is a
//   second tensor-core kernel (gz^T x shifted input, one GEMM per tap, the bias gradient as an
//   extra GEMM against ones) writing per-CTA partials that a fixed-order reduction sums.
// * Adam on the FP32 master weights, repacked to bfloat16 after every step.
// * A replay buffer of training pairs made from error samples of the Poisson operator.
//
// The network is small (16 channels) and each layer's data fits in L2, so the kernels are
// bounded by latency and issue rate rather than by HBM; they are written for few launches
// and no host synchronisation so that one application can be captured in a CUDA graph.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "reduce.cuh"

using bf16 = __nv_bfloat16;

namespace chns {
namespace lp {

constexpr int kC = 16;                        // channels
constexpr int kVS = 24;                       // shared-memory voxel stride (bf16): 48 bytes
constexpr int kTX = 8, kTY = 8, kTZ = 4;      // output tile of one CTA
constexpr int kTile = kTX * kTY * kTZ;        // 256 voxels = 16 M-tiles of 16
constexpr int kHX = kTX + 2, kHY = kTY + 2, kHZ = kTZ + 2;
constexpr int kHalo = kHX * kHY * kHZ;        // 600 voxels
constexpr int kThreads = 256;                 // 8 warps
constexpr int kWRows = 27 * kC;               // weight rows (tap, output channel)
constexpr int kConvSmem = (kHalo + kWRows) * kVS * 2;   // 49,536 bytes
constexpr int kWgSmem = (kHalo + kTile) * kVS * 2;      // 41,088 bytes
constexpr int kWgOut = 27 * kC * kC + kC;     // weight-gradient partial: 27x16x16 + bias 16
constexpr int kLayers = 7;                    // enc0..enc3, dec2, dec1, dec0
constexpr int kOutParts = 18;                 // out-layer partials: 16 W, 1 b, 1 loss
constexpr int kMaxParts = 2048;               // partial rows of the weight-gradient kernel

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void ldsm_x4(uint32_t a, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t a, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                          uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
// d += A (16x16, row) * B (16x8, col), bf16 inputs, fp32 accumulators
__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct TileXYZ {
  int x0, y0, z0;
};
__device__ __forceinline__ TileXYZ tile_origin(int tile, int D) {
  const int tx = (D + kTX - 1) / kTX, ty = (D + kTY - 1) / kTY;
  TileXYZ o;
  o.x0 = (tile % tx) * kTX;
  o.y0 = ((tile / tx) % ty) * kTY;
  o.z0 = (tile / (tx * ty)) * kTZ;
  return o;
}
__host__ __device__ inline int num_tiles(int D) {
  return ((D + kTX - 1) / kTX) * ((D + kTY - 1) / kTY) * ((D + kTZ - 1) / kTZ);
}
// voxel v of a tile (x fastest)
__device__ __forceinline__ void tile_voxel(int v, int& x, int& y, int& z) {
  x = v & (kTX - 1);
  y = (v / kTX) & (kTY - 1);
  z = v / (kTX * kTY);
}

// Stage the (kTX+2) x (kTY+2) x (kTZ+2) halo of a tile (zero outside the grid).
__device__ __forceinline__ void load_halo(const bf16* __restrict__ in, int D, TileXYZ o,
                                          bf16* hs) {
  for (int i = threadIdx.x; i < kHalo * 2; i += kThreads) {
    const int v = i >> 1, h = i & 1;
    const int hx = v % kHX, hy = (v / kHX) % kHY, hz = v / (kHX * kHY);
    const int gx = o.x0 - 1 + hx, gy = o.y0 - 1 + hy, gz = o.z0 - 1 + hz;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (gx >= 0 && gx < D && gy >= 0 && gy < D && gz >= 0 && gz < D)
      val = reinterpret_cast<const uint4*>(in)[((((int64_t)gz * D + gy) * D + gx) << 1) + h];
    *reinterpret_cast<uint4*>(hs + v * kVS + h * 8) = val;
  }
}

// ---------------------------------------------------------------- 3x3x3 convolution
// out[v][co] = sum_t sum_ci W[t][co][ci] in[v + d_t][ci] (+ bias, ReLU, bf16 store when FWD;
// linear FP32 store otherwise). Each warp computes two M-tiles of 16 voxels x 16 channels.
template <bool FWD>
__global__ void __launch_bounds__(kThreads)
k_conv(const bf16* __restrict__ in, const bf16* __restrict__ W, const float* __restrict__ bias,
       void* __restrict__ out, int D) {
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* hs = reinterpret_cast<bf16*>(smem);
  bf16* wsm = hs + kHalo * kVS;
  const TileXYZ o = tile_origin(blockIdx.x, D);
  for (int i = threadIdx.x; i < kWRows * 2; i += kThreads)
    *reinterpret_cast<uint4*>(wsm + (i >> 1) * kVS + (i & 1) * 8) =
        reinterpret_cast<const uint4*>(W)[i];
  load_halo(in, D, o, hs);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = lane >> 3, i8 = lane & 7;
  // ldmatrix row addresses: A (voxels x input channels): matrix j holds rows 8*(j&1).., channel
  // half j>>1; B (output channel rows x input channels): matrix j holds n-tile j>>1, half j&1.
  int abase[2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    int x, y, z;
    tile_voxel((warp * 2 + mt) * 16 + i8 + 8 * (j & 1), x, y, z);
    abase[mt] = ((z + 1) * kHY + (y + 1)) * kHX + (x + 1);
  }
  const uint32_t hs_a = smem_u32(hs) + (j >> 1) * 16;
  const uint32_t ws_a = smem_u32(wsm) + ((j >> 1) * 8 + i8) * (kVS * 2) + (j & 1) * 16;
  float acc[2][2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
#pragma unroll 3
  for (int t = 0; t < 27; ++t) {
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    const int sh = (dz * kHY + dy) * kHX + dx;
    uint32_t b0, b1, b2, b3;
    ldsm_x4(ws_a + t * kC * (kVS * 2), b0, b1, b2, b3);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      uint32_t a0, a1, a2, a3;
      ldsm_x4(hs_a + (abase[mt] + sh) * (kVS * 2), a0, a1, a2, a3);
      mma16816(acc[mt][0], a0, a1, a2, a3, b0, b1);
      mma16816(acc[mt][1], a0, a1, a2, a3, b2, b3);
    }
  }
  // epilogue: fragment rows gid / gid+8, columns 2*tq, 2*tq+1 of each n-tile
  const int gid = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      int x, y, z;
      tile_voxel((warp * 2 + mt) * 16 + gid + 8 * hf, x, y, z);
      x += o.x0;
      y += o.y0;
      z += o.z0;
      if (x >= D || y >= D || z >= D) continue;
      const int64_t vox = ((int64_t)z * D + y) * D + x;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int co = nt * 8 + 2 * tq;
        float v0 = acc[mt][nt][2 * hf], v1 = acc[mt][nt][2 * hf + 1];
        if (FWD) {
          v0 = fmaxf(v0 + bias[co], 0.f);
          v1 = fmaxf(v1 + bias[co + 1], 0.f);
          reinterpret_cast<__nv_bfloat162*>(out)[(vox * kC + co) >> 1] =
              __floats2bfloat162_rn(v0, v1);
        } else {
          reinterpret_cast<float2*>(out)[(vox * kC + co) >> 1] = make_float2(v0, v1);
        }
      }
    }
}

// First layer (2 input channels): the contraction index k = 2 tap + channel runs over 54 values,
// padded to 64 = 4 MMA k-steps instead of 27 (16 channels x 27 taps). A register holds the two
// channels of one voxel at one tap (one 32-bit shared load); B the two weights of one tap.
__global__ void __launch_bounds__(kThreads)
k_conv_c2(const __nv_bfloat162* __restrict__ in, const bf16* __restrict__ W,
          const float* __restrict__ bias, bf16* __restrict__ out, int D) {
  __shared__ uint32_t hs[kHalo];
  __shared__ uint32_t wsm[27 * kC];
  const TileXYZ o = tile_origin(blockIdx.x, D);
  for (int i = threadIdx.x; i < 27 * kC; i += kThreads)
    wsm[i] = reinterpret_cast<const uint32_t*>(W)[i * 8];  // W[tap][co][0..1]
  for (int v = threadIdx.x; v < kHalo; v += kThreads) {
    const int hx = v % kHX, hy = (v / kHX) % kHY, hz = v / (kHX * kHY);
    const int gx = o.x0 - 1 + hx, gy = o.y0 - 1 + hy, gz = o.z0 - 1 + hz;
    uint32_t val = 0u;
    if (gx >= 0 && gx < D && gy >= 0 && gy < D && gz >= 0 && gz < D)
      val = reinterpret_cast<const uint32_t*>(in)[((int64_t)gz * D + gy) * D + gx];
    hs[v] = val;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tq = lane & 3;
  int hrow[2][2];  // halo index of fragment rows gid and gid + 8 of each M-tile
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      int x, y, z;
      tile_voxel((warp * 2 + mt) * 16 + gid + 8 * hf, x, y, z);
      hrow[mt][hf] = ((z + 1) * kHY + (y + 1)) * kHX + (x + 1);
    }
  float acc[2][2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const int ta = kk * 8 + tq, tb = ta + 4;
    const bool va = ta < 27, vb = tb < 27;
    const int sa = va ? ((ta / 9 - 1) * kHY + (ta / 3) % 3 - 1) * kHX + ta % 3 - 1 : 0;
    const int sb = vb ? ((tb / 9 - 1) * kHY + (tb / 3) % 3 - 1) * kHX + tb % 3 - 1 : 0;
    uint32_t b[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      b[nt][0] = va ? wsm[ta * kC + nt * 8 + gid] : 0u;
      b[nt][1] = vb ? wsm[tb * kC + nt * 8 + gid] : 0u;
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const uint32_t a0 = va ? hs[hrow[mt][0] + sa] : 0u;
      const uint32_t a1 = va ? hs[hrow[mt][1] + sa] : 0u;
      const uint32_t a2 = vb ? hs[hrow[mt][0] + sb] : 0u;
      const uint32_t a3 = vb ? hs[hrow[mt][1] + sb] : 0u;
      mma16816(acc[mt][0], a0, a1, a2, a3, b[0][0], b[0][1]);
      mma16816(acc[mt][1], a0, a1, a2, a3, b[1][0], b[1][1]);
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      int x, y, z;
      tile_voxel((warp * 2 + mt) * 16 + gid + 8 * hf, x, y, z);
      x += o.x0;
      y += o.y0;
      z += o.z0;
      if (x >= D || y >= D || z >= D) continue;
      const int64_t vox = ((int64_t)z * D + y) * D + x;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int co = nt * 8 + 2 * tq;
        const float v0 = fmaxf(acc[mt][nt][2 * hf] + bias[co], 0.f);
        const float v1 = fmaxf(acc[mt][nt][2 * hf + 1] + bias[co + 1], 0.f);
        reinterpret_cast<__nv_bfloat162*>(out)[(vox * kC + co) >> 1] = __floats2bfloat162_rn(v0, v1);
      }
    }
}

// ---------------------------------------------------------------- weight gradient
// part[blk][t][co][ci] = sum over the voxels v of the CTA's tiles of gz[v][co] in[v + d_t][ci];
// part[blk][27*256 + co] = sum_v gz[v][co] (bias). GEMM per tap: M = co, N = ci, K = voxels,
// both operands from channel-last shared tiles through ldmatrix.trans.
__global__ void __launch_bounds__(kThreads)
k_wgrad(const bf16* __restrict__ in, const bf16* __restrict__ gz, int D, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* hs = reinterpret_cast<bf16*>(smem);
  bf16* gs = hs + kHalo * kVS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = lane >> 3, i8 = lane & 7;
  // taps of this warp: warp + 8 s for s = 0..3 (< 27); warp 7's fourth slot is the bias
  float acc[4][2][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const uint32_t ones = 0x3F803F80u;  // two bfloat16 1.0
  const int ntiles = ((D + kTX - 1) / kTX) * ((D + kTY - 1) / kTY) * ((D + kTZ - 1) / kTZ);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const TileXYZ o = tile_origin(tile, D);
    __syncthreads();
    load_halo(in, D, o, hs);
    for (int i = threadIdx.x; i < kTile * 2; i += kThreads) {
      const int v = i >> 1, h = i & 1;
      int x, y, z;
      tile_voxel(v, x, y, z);
      x += o.x0;
      y += o.y0;
      z += o.z0;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (x < D && y < D && z < D)
        val = reinterpret_cast<const uint4*>(gz)[((((int64_t)z * D + y) * D + x) << 1) + h];
      *reinterpret_cast<uint4*>(gs + v * kVS + h * 8) = val;
    }
    __syncthreads();
#pragma unroll 1
    for (int ks = 0; ks < kTile / 16; ++ks) {
      // A = gz^T (16 co x 16 voxels): matrix j holds voxels 8*(j>>1).., channel half j&1
      uint32_t a0, a1, a2, a3;
      ldsm_x4_t(smem_u32(gs + (ks * 16 + i8 + 8 * (j >> 1)) * kVS + (j & 1) * 8), a0, a1, a2, a3);
      // B row addresses: matrix j holds voxels 8*(j&1).., channel half j>>1
      int x, y, z;
      tile_voxel(ks * 16 + i8 + 8 * (j & 1), x, y, z);
      const int hb = ((z + 1) * kHY + (y + 1)) * kHX + (x + 1);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int t = warp + 8 * s;
        if (t < 27) {
          const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
          const int hv = hb + (dz * kHY + dy) * kHX + dx;
          uint32_t b0, b1, b2, b3;
          ldsm_x4_t(smem_u32(hs + hv * kVS + (j >> 1) * 8), b0, b1, b2, b3);
          mma16816(acc[s][0], a0, a1, a2, a3, b0, b1);
          mma16816(acc[s][1], a0, a1, a2, a3, b2, b3);
        } else if (s == 3 && warp == 7) {
          mma16816(acc[3][0], a0, a1, a2, a3, ones, ones);
        }
      }
    }
  }
  float* pb = part + (int64_t)blockIdx.x * kWgOut;
  const int gid = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int t = warp + 8 * s;
    if (t < 27) {
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int ci = nt * 8 + 2 * tq;
        pb[t * 256 + gid * 16 + ci] = acc[s][nt][0];
        pb[t * 256 + gid * 16 + ci + 1] = acc[s][nt][1];
        pb[t * 256 + (gid + 8) * 16 + ci] = acc[s][nt][2];
        pb[t * 256 + (gid + 8) * 16 + ci + 1] = acc[s][nt][3];
      }
    } else if (s == 3 && warp == 7 && tq == 0) {
      pb[27 * 256 + gid] = acc[3][0][0];
      pb[27 * 256 + gid + 8] = acc[3][0][2];
    }
  }
}

// Sum the partial rows in a fixed order into the flat gradient of one layer (cin input
// channels of the 16 computed).
__global__ void k_wgrad_reduce(const float* __restrict__ part, int nparts, int cin,
                               float* __restrict__ gW, float* __restrict__ gb) {
  const int nw = 27 * kC * cin;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nw + kC) return;
  int src;
  if (o < nw) {
    const int t = o / (kC * cin), co = (o / cin) % kC, ci = o % cin;
    src = t * 256 + co * 16 + ci;
  } else {
    src = 27 * 256 + (o - nw);
  }
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += (double)part[(int64_t)p * kWgOut + src];
  if (o < nw) gW[o] = (float)s;
  else gb[o - nw] = (float)s;
}

// ---------------------------------------------------------------- pooling, skip, output layer
// out (Dc^3) = mean of the 8 children of in (2 Dc); one thread per (voxel, 8-channel half)
__global__ void k_pool(const bf16* __restrict__ in, bf16* __restrict__ out, int Dc) {
  const int64_t n = (int64_t)Dc * Dc * Dc * 2;
  const int Df = 2 * Dc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(i & 1);
    const int64_t v = i >> 1;
    const int x = (int)(v % Dc), y = (int)((v / Dc) % Dc), z = (int)(v / ((int64_t)Dc * Dc));
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t fv = ((int64_t)(2 * z + (c >> 2)) * Df + 2 * y + ((c >> 1) & 1)) * Df +
                         2 * x + (c & 1);
      const uint4 u = reinterpret_cast<const uint4*>(in)[(fv << 1) + h];
      const __nv_bfloat162* p = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(p[k]);
        s[2 * k] += f.x;
        s[2 * k + 1] += f.y;
      }
    }
    uint4 r;
    __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = __floats2bfloat162_rn(s[2 * k] * 0.125f, s[2 * k + 1] * 0.125f);
    reinterpret_cast<uint4*>(out)[i] = r;
  }
}

// out (Df^3) = up(coarse) + skip
__global__ void k_upadd(const bf16* __restrict__ coarse, const bf16* __restrict__ skip,
                        bf16* __restrict__ out, int Df) {
  const int64_t n = (int64_t)Df * Df * Df * 2;
  const int Dc = Df / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(i & 1);
    const int64_t v = i >> 1;
    const int x = (int)(v % Df), y = (int)((v / Df) % Df), z = (int)(v / ((int64_t)Df * Df));
    const int64_t cv = ((int64_t)(z >> 1) * Dc + (y >> 1)) * Dc + (x >> 1);
    const uint4 a = reinterpret_cast<const uint4*>(coarse)[(cv << 1) + h];
    const uint4 b = reinterpret_cast<const uint4*>(skip)[i];
    const __nv_bfloat162* pa = reinterpret_cast<const __nv_bfloat162*>(&a);
    const __nv_bfloat162* pb = reinterpret_cast<const __nv_bfloat162*>(&b);
    uint4 r;
    __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 fa = __bfloat1622float2(pa[k]), fb = __bfloat1622float2(pb[k]);
      q[k] = __floats2bfloat162_rn(fa.x + fb.x, fa.y + fb.y);
    }
    reinterpret_cast<uint4*>(out)[i] = r;
  }
}

__device__ __forceinline__ void load16(const bf16* p, int64_t v, float (&f)[16]) {
  const uint4* q = reinterpret_cast<const uint4*>(p) + (v << 1);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint4 u = q[h];
    const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 t = __bfloat1622float2(b[k]);
      f[h * 8 + 2 * k] = t.x;
      f[h * 8 + 2 * k + 1] = t.y;
    }
  }
}

// out[v] = sum_c w[c] d0[v][c] + b  (w = P + offset: 16 weights then the bias)
__global__ void k_outconv(const bf16* __restrict__ d0, const float* __restrict__ w,
                          float* __restrict__ out, int64_t nv) {
  __shared__ float sw[kC + 1];
  if (threadIdx.x <= kC) sw[threadIdx.x] = w[threadIdx.x];
  __syncthreads();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    float f[16];
    load16(d0, v, f);
    float s = sw[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) s = fmaf(sw[c], f[c], s);
    out[v] = s;
  }
}

// Output-layer backward (and the loss): gout = (out - target * inv_ts) / nv when a target is
// given, else gout_in; gz[v][c] = bf16(w[c] gout (d0[v][c] > 0)); per-block partials of
// sum gout d0[c] (16), sum gout, sum (out - target * inv_ts)^2.
__global__ void __launch_bounds__(kThreads)
k_out_bwd(const float* __restrict__ out, const float* __restrict__ target, float inv_ts,
          const float* __restrict__ gout_in, const bf16* __restrict__ d0,
          const float* __restrict__ w, bf16* __restrict__ gz, float* __restrict__ part,
          int64_t nv) {
  __shared__ float sw[kC];
  if (threadIdx.x < kC) sw[threadIdx.x] = w[threadIdx.x];
  __syncthreads();
  const float inv_n = 1.0f / (float)nv;
  double acc[kOutParts];
#pragma unroll
  for (int k = 0; k < kOutParts; ++k) acc[k] = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    float g, d2 = 0.f;
    if (target) {
      const float diff = out[v] - target[v] * inv_ts;
      g = diff * inv_n;
      d2 = diff * diff;
    } else {
      g = gout_in[v];
    }
    float f[16];
    load16(d0, v, f);
    uint4 r[2];
    __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(r);
#pragma unroll
    for (int c = 0; c < kC; c += 2) {
      const float z0 = f[c] > 0.f ? sw[c] * g : 0.f;
      const float z1 = f[c + 1] > 0.f ? sw[c + 1] * g : 0.f;
      q[c >> 1] = __floats2bfloat162_rn(z0, z1);
      acc[c] += (double)(g * f[c]);
      acc[c + 1] += (double)(g * f[c + 1]);
    }
    reinterpret_cast<uint4*>(gz)[v << 1] = r[0];
    reinterpret_cast<uint4*>(gz)[(v << 1) + 1] = r[1];
    acc[16] += (double)g;
    acc[17] += (double)d2;
  }
  double tot[kOutParts];
  block_sum<kOutParts, kThreads>(acc, tot);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < kOutParts; ++k) part[(int64_t)blockIdx.x * kOutParts + k] = (float)tot[k];
}

// G[out.W] (16), G[out.b] and loss = sum d^2 / (2 nv) from the partial rows
__global__ void k_out_reduce(const float* __restrict__ part, int nparts, float* __restrict__ g,
                             float* __restrict__ loss, int64_t nv) {
  const int k = threadIdx.x;
  if (k >= kOutParts) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += (double)part[p * kOutParts + k];
  if (k < 17) g[k] = (float)s;
  else if (loss) *loss = (float)(0.5 * s / (double)nv);
}

// gz[v][c] = bf16((up_backward(gA)[v] + gB[v] + gC[parent(v)] / 8)[c] (relu_out[v][c] > 0));
// gA at 2D (sum of the 8 children), gB at D, gC at D/2; any of them may be null.
__global__ void k_mask(const float* __restrict__ gA, const float* __restrict__ gB,
                       const float* __restrict__ gC, const bf16* __restrict__ relu_out,
                       bf16* __restrict__ gz, int D) {
  const int64_t n = (int64_t)D * D * D * 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(i & 1);
    const int64_t v = i >> 1;
    const int x = (int)(v % D), y = (int)((v / D) % D), z = (int)(v / ((int64_t)D * D));
    float g[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (gA) {
      const int Df = 2 * D;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t fv = ((int64_t)(2 * z + (c >> 2)) * Df + 2 * y + ((c >> 1) & 1)) * Df +
                           2 * x + (c & 1);
        const float4* p = reinterpret_cast<const float4*>(gA + fv * kC + h * 8);
        const float4 a = p[0], b = p[1];
        g[0] += a.x; g[1] += a.y; g[2] += a.z; g[3] += a.w;
        g[4] += b.x; g[5] += b.y; g[6] += b.z; g[7] += b.w;
      }
    }
    if (gB) {
      const float4* p = reinterpret_cast<const float4*>(gB + v * kC + h * 8);
      const float4 a = p[0], b = p[1];
      g[0] += a.x; g[1] += a.y; g[2] += a.z; g[3] += a.w;
      g[4] += b.x; g[5] += b.y; g[6] += b.z; g[7] += b.w;
    }
    if (gC) {
      const int Dc = D / 2;
      const int64_t cv = ((int64_t)(z >> 1) * Dc + (y >> 1)) * Dc + (x >> 1);
      const float4* p = reinterpret_cast<const float4*>(gC + cv * kC + h * 8);
      const float4 a = p[0], b = p[1];
      g[0] += 0.125f * a.x; g[1] += 0.125f * a.y; g[2] += 0.125f * a.z; g[3] += 0.125f * a.w;
      g[4] += 0.125f * b.x; g[5] += 0.125f * b.y; g[6] += 0.125f * b.z; g[7] += 0.125f * b.w;
    }
    const uint4 u = reinterpret_cast<const uint4*>(relu_out)[i];
    const __nv_bfloat162* o = reinterpret_cast<const __nv_bfloat162*>(&u);
    uint4 r;
    __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __bfloat1622float2(o[k]);
      q[k] = __floats2bfloat162_rn(f.x > 0.f ? g[2 * k] : 0.f, f.y > 0.f ? g[2 * k + 1] : 0.f);
    }
    reinterpret_cast<uint4*>(gz)[i] = r;
  }
}

// ---------------------------------------------------------------- parameters
struct Offsets {
  int w[kLayers], b[kLayers], cin[kLayers];
  int outw, total;
};
inline Offsets make_offsets() {
  Offsets o{};
  int p = 0;
  for (int k = 0; k < kLayers; ++k) {
    o.cin[k] = k == 0 ? 2 : kC;
    o.w[k] = p;
    p += 27 * kC * o.cin[k];
    o.b[k] = p;
    p += kC;
  }
  o.outw = p;
  p += kC + 1;
  o.total = p;
  return o;
}

// Wf[k][t][co][ci] = bf16(W_k[t][co][ci]) (ci >= cin: 0);
// Wt[k][t][ci][co] = Wf[k][26 - t][co][ci] (the transposed convolution of the backward pass)
__global__ void k_pack(const float* __restrict__ P, Offsets o, bf16* __restrict__ Wf,
                       bf16* __restrict__ Wt) {
  const int n = kLayers * 27 * 256;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = i / (27 * 256), r = i % (27 * 256);
    const int t = r / 256, co = (r / 16) % 16, ci = r % 16;
    const int cin = o.cin[k];
    const bf16 w = __float2bfloat16_rn(ci < cin ? P[o.w[k] + (t * kC + co) * cin + ci] : 0.f);
    Wf[i] = w;
    Wt[k * 27 * 256 + (26 - t) * 256 + ci * 16 + co] = w;
  }
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float ibc1, float ibc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi * ibc1) / (sqrtf(vi * ibc2) + eps);
  }
}

// ---------------------------------------------------------------- grid transfer
// Trilinear weights of node i: base cell (i0, j0, k0) and fractions t (constant extrapolation
// beyond the outermost centres). With D a power of two the coordinates are exact in FP32.
struct Tri {
  int i0[3];
  float t[3];
};
__device__ __forceinline__ Tri trilinear(const uint32_t* __restrict__ xyz, int64_t i, int D,
                                         float scale) {
  Tri w;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float s = (float)xyz[3 * i + d] * scale - 0.5f;
    int a = (int)floorf(s);
    a = min(max(a, 0), D - 2);
    w.i0[d] = a;
    w.t[d] = fminf(fmaxf(s - (float)a, 0.f), 1.f);
  }
  return w;
}
__device__ __forceinline__ float tri_w(const Tri& w, int c) {
  return ((c & 1) ? w.t[0] : 1.f - w.t[0]) * ((c & 2) ? w.t[1] : 1.f - w.t[1]) *
         ((c & 4) ? w.t[2] : 1.f - w.t[2]);
}
__device__ __forceinline__ int64_t tri_cell(const Tri& w, int c, int D) {
  return ((int64_t)(w.i0[2] + ((c >> 2) & 1)) * D + (w.i0[1] + ((c >> 1) & 1))) * D +
         (w.i0[0] + (c & 1));
}

// grid += R f  (and wsum += R 1 when wsum is given); f = log(1/rho(clamp(phi))) when logrho
template <class T>
__global__ void k_restrict(const T* __restrict__ f, const uint32_t* __restrict__ xyz, int64_t N,
                           int D, float scale, float* __restrict__ grid, float* __restrict__ wsum,
                           bool logrho, float alpha, float beta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v = (float)f[i];
    if (logrho) v = -logf(alpha * fminf(fmaxf(v, -1.f), 1.f) + beta);
    const Tri w = trilinear(xyz, i, D, scale);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float wc = tri_w(w, c);
      const int64_t cell = tri_cell(w, c, D);
      atomicAdd(grid + cell, wc * v);
      if (wsum) atomicAdd(wsum + cell, wc);
    }
  }
}

// a[c] = wsum[c] > 0 ? a[c] / wsum[c] : 0
__global__ void k_cell_mean(float* __restrict__ a, const float* __restrict__ wsum, int64_t n,
                            float extra_scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float w = wsum[i];
    a[i] = w > 0.f ? a[i] / w * extra_scale : 0.f;
  }
}

// 1/s from r.r (device) or from a host value; s = sqrt(r.r / nv)
__device__ __forceinline__ float inv_scale(const double* rr, float inv_s_host, float inv_nv) {
  if (!rr) return inv_s_host;
  const float q = (float)(*rr) * inv_nv;
  return q > 0.f ? rsqrtf(q) : 0.f;
}

// x2[v] = (bf16(gr[v] / s), bf16(lr[v])); x16 (optional): the same as 16 channels, zero-padded
__device__ __forceinline__ void put_input(__nv_bfloat162 v2, int64_t v, __nv_bfloat162* x2,
                                          bf16* x16) {
  x2[v] = v2;
  if (x16) {
    uint4 r0 = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<__nv_bfloat162*>(&r0.x) = v2;
    reinterpret_cast<uint4*>(x16)[v << 1] = r0;
    reinterpret_cast<uint4*>(x16)[(v << 1) + 1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

__global__ void k_pack_input(const float* __restrict__ gr, const float* __restrict__ lr,
                             const double* __restrict__ rr, float inv_s_host, float inv_nv,
                             __nv_bfloat162* __restrict__ x2, bf16* __restrict__ x16, int64_t nv) {
  const float is = inv_scale(rr, inv_s_host, inv_nv);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x)
    put_input(__floats2bfloat162_rn(gr[v] * is, lr[v]), v, x2, x16);
}

// planar FP32 (2, D^3) -> bf16 inputs
__global__ void k_pack_planar(const float* __restrict__ x, __nv_bfloat162* __restrict__ x2,
                              bf16* __restrict__ x16, int64_t nv) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x)
    put_input(__floats2bfloat162_rn(x[v], x[nv + v]), v, x2, x16);
}

// replay pair k: (x (2 bf16 per voxel), target FP32)
__global__ void k_store_pair(const float* __restrict__ gr, const float* __restrict__ lr,
                             float inv_s, __nv_bfloat162* __restrict__ xs, int64_t nv) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x)
    xs[v] = __floats2bfloat162_rn(gr[v] * inv_s, lr[v]);
}
__global__ void k_load_pair(const __nv_bfloat162* __restrict__ xs, __nv_bfloat162* __restrict__ x2,
                            bf16* __restrict__ x16, int64_t nv) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x)
    put_input(xs[v], v, x2, x16);
}
// z[i] = (dinv ? dinv[i] r[i] : 0) + s out_scale sum_c w_c grid[cell_c]  (s = 1 without rr)
template <class T>
__global__ void k_prolong(const float* __restrict__ grid, const uint32_t* __restrict__ xyz,
                          int64_t N, int D, float scale, const double* __restrict__ rr,
                          float inv_nv, float out_scale, const T* __restrict__ dinv,
                          const T* __restrict__ r, T* __restrict__ z) {
  float sc = out_scale;
  if (rr) {
    const float q = (float)(*rr) * inv_nv;
    sc *= q > 0.f ? sqrtf(q) : 0.f;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Tri w = trilinear(xyz, i, D, scale);
    float c = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) c = fmaf(tri_w(w, k), grid[tri_cell(w, k, D)], c);
    T out = (T)(sc * c);
    if (dinv) out += dinv[i] * r[i];
    z[i] = out;
  }
}

// d[i] = e[i] - sc sum_c w_c grid[cell_c]  (the error left by the correction, FP32)
__global__ void k_prolong_diff(const float* __restrict__ grid, const uint32_t* __restrict__ xyz,
                               int64_t N, int D, float scale, float sc, const float* __restrict__ e,
                               float* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Tri w = trilinear(xyz, i, D, scale);
    float c = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) c = fmaf(tri_w(w, k), grid[tri_cell(w, k, D)], c);
    d[i] = e[i] - sc * c;
  }
}

// *out += f * (a . b) (block sums in FP64, one float atomic per block)
__global__ void __launch_bounds__(kThreads)
k_dot_acc(const float* __restrict__ a, const float* __restrict__ b, int64_t n, float f,
          float* __restrict__ out) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[0] += (double)a[i] * (double)b[i];
  double t[1];
  block_sum<1, kThreads>(v, t);
  if (threadIdx.x == 0) atomicAdd(out, (float)(f * t[0]));
}

__global__ void k_scale_f(const float* __restrict__ a, float* __restrict__ b, int64_t n, float f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i] * f;
}

// b = a f / max(1, *loss): a pair whose correction makes the error worse than no correction
// (relative energy above 1) contributes a gradient of bounded size (that of log(loss))
__global__ void k_scale_grad(const float* __restrict__ a, float* __restrict__ b, int64_t n, float f,
                             const float* __restrict__ loss) {
  const float g = f / fmaxf(1.f, *loss);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i] * g;
}

__global__ void k_square_sum(const float* __restrict__ a, int64_t n, double* __restrict__ part) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[0] += (double)a[i] * (double)a[i];
  double t[1];
  block_sum<1, kThreads>(v, t);
  if (threadIdx.x == 0) part[blockIdx.x] = t[0];
}

inline unsigned grid_for(int64_t n, int threads = kThreads) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 4096));
}

uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace lp
}  // namespace chns

using namespace chns;
using namespace chns::lp;

struct chns_learned {
  int D = 0;
  int64_t nv = 0;          // D^3
  int capacity = 0, count = 0, next = 0;
  Offsets off{};
  double out_scale = 0.0;  // 0: not set
  int adam_t = 0;
  int sm_count = 0;
  // parameters (FP32) and training state
  float *P = nullptr, *G = nullptr, *Am = nullptr, *Av = nullptr;
  bf16 *Wf = nullptr, *Wt = nullptr;
  // activations (bf16 channel-last, 16 channels); level l has (D >> l)^3 voxels
  bf16* x0 = nullptr;            // input, 16 channels (zero-padded; weight gradient of enc0)
  __nv_bfloat162* x2 = nullptr;  // input, 2 channels (forward)
  bf16* enc[4] = {};
  bf16* ein[4] = {};   // pooled inputs of enc1..enc3
  bf16* din[3] = {};   // inputs of dec0..dec2
  bf16* dec[3] = {};
  float* out = nullptr;  // D^3
  // backward
  bf16* gz = nullptr;
  float* gdec[3] = {};   // gradient with respect to the input of dec_l (level l)
  float* gein[4] = {};   // gradient with respect to the input of enc_l (level l, l >= 1)
  float* wpart = nullptr;   // weight-gradient partial rows
  float* opart = nullptr;   // output-layer partial rows
  int wparts = 0, oparts = 0;
  // grid scratch
  float *g_r = nullptr, *g_lr = nullptr, *g_w = nullptr, *g_t = nullptr;
  double* dscal = nullptr;  // device scalars
  // replay buffer: grid inputs and targets; per pair the mean-free error e (FP32) and the
  // coefficient 1 + phi~ (bfloat16) on the nodes of the bound mesh, s(A e) and e^T A e
  __nv_bfloat162* rx = nullptr;
  float* rt = nullptr;
  const chns_mesh* bound = nullptr;
  int64_t bound_n = 0;
  float* re = nullptr;
  bf16* rphi = nullptr;
  float *d32 = nullptr, *w32 = nullptr;
  std::vector<double> hs, heae;
  float* loss_dev = nullptr;
  int loss_cap = 0;
};

namespace chns {
namespace lp {

static bool conv_attr_done = false;

static chns_status set_attrs() {
  if (conv_attr_done) return CHNS_OK;
  CHNS_CUDA(cudaFuncSetAttribute(k_conv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem));
  CHNS_CUDA(cudaFuncSetAttribute(k_conv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem));
  CHNS_CUDA(cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem));
  conv_attr_done = true;
  return CHNS_OK;
}

static int lvl(const chns_learned* L, int l) { return L->D >> l; }
static int64_t vox(const chns_learned* L, int l) {
  const int64_t d = lvl(L, l);
  return d * d * d;
}

static void conv(const chns_learned* L, bool fwd, const bf16* in, int layer, void* out, int D,
                 cudaStream_t s) {
  const bf16* W = (fwd ? L->Wf : L->Wt) + (size_t)layer * 27 * 256;
  note_launch();
  if (fwd)
    k_conv<true><<<num_tiles(D), kThreads, kConvSmem, s>>>(in, W, L->P + L->off.b[layer], out, D);
  else
    k_conv<false><<<num_tiles(D), kThreads, kConvSmem, s>>>(in, W, nullptr, out, D);
}

static void wgrad(chns_learned* L, const bf16* in, int layer, int D, cudaStream_t s) {
  const int nt = num_tiles(D);
  const int parts = std::min(nt, L->wparts);
  note_launch();
  k_wgrad<<<parts, kThreads, kWgSmem, s>>>(in, L->gz, D, L->wpart);
  const int nout = 27 * kC * L->off.cin[layer] + kC;
  note_launch();
  k_wgrad_reduce<<<(nout + 255) / 256, 256, 0, s>>>(L->wpart, parts, L->off.cin[layer],
                                                     L->G + L->off.w[layer], L->G + L->off.b[layer]);
}

// Forward pass from L->x2; output in L->out.
static chns_status forward(chns_learned* L, cudaStream_t s) {
  note_launch();
  k_conv_c2<<<num_tiles(L->D), kThreads, 0, s>>>(L->x2, L->Wf, L->P + L->off.b[0], L->enc[0], L->D);
  for (int l = 1; l < 4; ++l) {
    note_launch();
    k_pool<<<grid_for(vox(L, l) * 2), kThreads, 0, s>>>(L->enc[l - 1], L->ein[l], lvl(L, l));
    conv(L, true, L->ein[l], l, L->enc[l], lvl(L, l), s);
  }
  for (int l = 2; l >= 0; --l) {
    const bf16* coarse = l == 2 ? L->enc[3] : L->dec[l + 1];
    note_launch();
    k_upadd<<<grid_for(vox(L, l) * 2), kThreads, 0, s>>>(coarse, L->enc[l], L->din[l], lvl(L, l));
    conv(L, true, L->din[l], 6 - l, L->dec[l], lvl(L, l), s);
  }
  note_launch();
  k_outconv<<<grid_for(L->nv), kThreads, 0, s>>>(L->dec[0], L->P + L->off.outw, L->out, L->nv);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

// Backward pass of the last forward; fills L->G. target (with 1/out_scale) or gout.
static chns_status backward(chns_learned* L, const float* target, float inv_ts, const float* gout,
                            float* loss_slot, cudaStream_t s) {
  note_launch();
  k_out_bwd<<<L->oparts, kThreads, 0, s>>>(L->out, target, inv_ts, gout, L->dec[0],
                                           L->P + L->off.outw, L->gz, L->opart, L->nv);
  note_launch();
  k_out_reduce<<<1, 32, 0, s>>>(L->opart, L->oparts, L->G + L->off.outw, loss_slot, L->nv);
  // decoder: dec0, dec1, dec2
  for (int l = 0; l < 3; ++l) {
    if (l > 0) {
      note_launch();
      k_mask<<<grid_for(vox(L, l) * 2), kThreads, 0, s>>>(L->gdec[l - 1], nullptr, nullptr,
                                                         L->dec[l], L->gz, lvl(L, l));
    }
    wgrad(L, L->din[l], 6 - l, lvl(L, l), s);
    conv(L, false, L->gz, 6 - l, L->gdec[l], lvl(L, l), s);
  }
  // encoder: enc3 .. enc0
  for (int l = 3; l >= 0; --l) {
    const float* gA = l == 3 ? L->gdec[2] : nullptr;
    const float* gB = l < 3 ? L->gdec[l] : nullptr;
    const float* gC = l < 3 ? L->gein[l + 1] : nullptr;
    note_launch();
    k_mask<<<grid_for(vox(L, l) * 2), kThreads, 0, s>>>(gA, gB, gC, L->enc[l], L->gz, lvl(L, l));
    wgrad(L, l == 0 ? L->x0 : L->ein[l], l, lvl(L, l), s);
    if (l > 0) conv(L, false, L->gz, l, L->gein[l], lvl(L, l), s);
  }
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

static void pack(chns_learned* L, cudaStream_t s) {
  note_launch();
  k_pack<<<grid_for(kLayers * 27 * 256), kThreads, 0, s>>>(L->P, L->off, L->Wf, L->Wt);
}

static void adam(chns_learned* L, const float* g, double lr, cudaStream_t s) {
  L->adam_t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const double bc1 = 1.0 - std::pow(b1, L->adam_t), bc2 = 1.0 - std::pow(b2, L->adam_t);
  note_launch();
  k_adam<<<grid_for(L->off.total), kThreads, 0, s>>>(L->P, g, L->Am, L->Av, L->off.total,
                                                      (float)lr, (float)b1, (float)b2, 1e-8f,
                                                      (float)(1.0 / bc1), (float)(1.0 / bc2));
  pack(L, s);
}

static float grid_scale(int D) { return std::ldexp((float)D, -CHNS_MAXD); }

// L->g_lr = cell mean of log(1/rho(clamp(phi~))); L->g_w = P_g^T 1
static chns_status density_channel(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                                   const chns_coef* coef, cudaStream_t s) {
  CHNS_CHECK(coef && coef->phi_tilde, CHNS_EINVAL, "learned: coefficient phi~ missing");
  const double rm = 1.0 / prm->rho_ratio;
  const float alpha = (float)((1.0 - rm) / 2.0), beta = (float)((1.0 + rm) / 2.0);
  CHNS_CUDA(cudaMemsetAsync(L->g_lr, 0, L->nv * sizeof(float), s));
  CHNS_CUDA(cudaMemsetAsync(L->g_w, 0, L->nv * sizeof(float), s));
  const int64_t N = m->d.n_nodes;
  note_launch();
  k_restrict<double><<<grid_for(N), kThreads, 0, s>>>(static_cast<const double*>(coef->phi_tilde),
                                                      m->d_node_int, N, L->D, grid_scale(L->D),
                                                      L->g_lr, L->g_w, true, alpha, beta);
  note_launch();
  k_cell_mean<<<grid_for(L->nv), kThreads, 0, s>>>(L->g_lr, L->g_w, L->nv, 1.0f);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

template <class T>
static void restrict_to(chns_learned* L, const chns_mesh* m, const T* r, float* grid,
                        cudaStream_t s) {
  cudaMemsetAsync(grid, 0, L->nv * sizeof(float), s);
  const int64_t N = m->d.n_nodes;
  note_launch();
  k_restrict<T><<<grid_for(N), kThreads, 0, s>>>(r, m->d_node_int, N, L->D, grid_scale(L->D),
                                                 grid, nullptr, false, 0.f, 0.f);
}

// host value of sum a^2 (FP32 grid or FP64 nodal via dot_host)
static chns_status grid_sq(chns_learned* L, const float* a, double* out, cudaStream_t s) {
  const unsigned nb = std::min<unsigned>(grid_for(L->nv), 1024);
  note_launch();
  k_square_sum<<<nb, kThreads, 0, s>>>(a, L->nv, L->dscal + 8);
  std::vector<double> h(nb);
  CHNS_CUDA(cudaMemcpyAsync(h.data(), L->dscal + 8, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  CHNS_CUDA(cudaStreamSynchronize(s));
  double t = 0.0;
  for (double v : h) t += v;
  *out = t;
  return CHNS_OK;
}

}  // namespace lp

// ---- hooks used by the Krylov solver (declared in internal.h)
chns_status learned_begin_solve(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                                const chns_coef* coef64, cudaStream_t s) {
  CHNS_CHECK(L, CHNS_EINVAL, "CHNS_PC_LEARNED needs solver_params.learned");
  CHNS_CHECK(L->out_scale > 0.0, CHNS_EINVAL, "learned: output scale not set (train first)");
  return lp::density_channel(L, m, prm, coef64, s);
}

template <class T>
chns_status learned_precondition(chns_learned* L, const chns_mesh* m, const T* r, const T* dinv,
                                 const double* rr_dev, T* z, cudaStream_t s) {
  using namespace lp;
  restrict_to<T>(L, m, r, L->g_r, s);
  const float inv_nv = (float)(1.0 / (double)L->nv);
  note_launch();
  k_pack_input<<<grid_for(L->nv), kThreads, 0, s>>>(L->g_r, L->g_lr, rr_dev, 0.f, inv_nv, L->x2,
                                                    nullptr, L->nv);
  chns_status st = forward(L, s);
  if (st != CHNS_OK) return st;
  const int64_t N = m->d.n_nodes;
  note_launch();
  k_prolong<T><<<grid_for(N), kThreads, 0, s>>>(L->out, m->d_node_int, N, L->D, grid_scale(L->D),
                                                rr_dev, inv_nv, (float)L->out_scale, dinv, r, z);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}
template chns_status learned_precondition<float>(chns_learned*, const chns_mesh*, const float*,
                                                 const float*, const double*, float*, cudaStream_t);
template chns_status learned_precondition<double>(chns_learned*, const chns_mesh*, const double*,
                                                  const double*, const double*, double*,
                                                  cudaStream_t);

chns_status learned_add_sample(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                               const chns_coef* coef, const double* e, cudaStream_t s) {
  using namespace lp;
  CHNS_CHECK(L && m && prm && coef && e, CHNS_EINVAL, "chns_learned_add_sample: null argument");
  CHNS_CHECK(L->capacity > 0, CHNS_EINVAL, "chns_learned_add_sample: no replay buffer");
  CHNS_CHECK(coef->phi_tilde, CHNS_EINVAL, "chns_learned_add_sample: coefficient phi~ missing");
  const int64_t N = m->d.n_nodes;
  if (!L->bound) {  // the nodal part of the replay buffer is sized for the first mesh
    const size_t cap = (size_t)L->capacity;
    if (cudaMalloc(&L->re, cap * N * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&L->rphi, cap * N * sizeof(bf16)) != cudaSuccess ||
        cudaMalloc(&L->d32, N * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&L->w32, N * sizeof(float)) != cudaSuccess) {
      set_error("chns_learned_add_sample: device allocation of the replay buffer failed");
      return CHNS_ENOMEM;
    }
    L->bound = m;
    L->bound_n = N;
  }
  CHNS_CHECK(L->bound == m && L->bound_n == N, CHNS_EINVAL,
             "chns_learned_add_sample: the replay buffer holds pairs of another mesh");
  double* r = nullptr;
  double* ep = nullptr;
  CHNS_CUDA(cudaMallocAsync(&r, N * sizeof(double), s));
  CHNS_CUDA(cudaMallocAsync(&ep, N * sizeof(double), s));
  // the error sample without its nodal mean: constants are the Poisson operator's null space, so
  // r = A e carries no information about them (and the solver returns mean-free iterates)
  double esum = 0.0;
  chns_status st = sum_host(m, e, N, &esum, s);
  if (st == CHNS_OK) {
    vec_copy(e, ep, N, s);
    CHNS_CUDA(cudaMemcpyAsync(L->dscal, &esum, sizeof(double), cudaMemcpyHostToDevice, s));
    vec_add_scalar(ep, L->dscal, -1.0 / (double)N, N, s);
    st = apply_op(m, CHNS_OP_POISSON, prm, coef, ep, r, CHNS_FP64, s);
  }
  double rr = 0.0;
  if (st == CHNS_OK) st = dot_host(m, r, r, N, &rr, s);
  if (st == CHNS_OK && rr > 0.0 && std::isfinite(rr)) {
    const double sc = std::sqrt(rr / (double)L->nv);
    st = density_channel(L, m, prm, coef, s);
    if (st == CHNS_OK) {
      restrict_to<double>(L, m, r, L->g_r, s);
      const int k = L->next;
      note_launch();
      k_store_pair<<<grid_for(L->nv), kThreads, 0, s>>>(L->g_r, L->g_lr, (float)(1.0 / sc),
                                                        L->rx + (size_t)k * L->nv, L->nv);
      float* t = L->rt + (size_t)k * L->nv;
      restrict_to<double>(L, m, ep, t, s);
      note_launch();
      k_cell_mean<<<grid_for(L->nv), kThreads, 0, s>>>(t, L->g_w, L->nv, (float)(1.0 / sc));
      double eae = 0.0;
      st = dot_host(m, ep, r, N, &eae, s);
      vec_convert_f64_f32(ep, L->re + (size_t)k * N, N, s);
      vec_convert_f64_bf16(static_cast<const double*>(coef->phi_tilde), L->rphi + (size_t)k * N, N,
                           1.0, s);
      L->hs[k] = sc;
      L->heae[k] = eae;
      L->next = (k + 1) % L->capacity;
      L->count = std::min(L->count + 1, L->capacity);
    }
  }
  cudaFreeAsync(r, s);
  cudaFreeAsync(ep, s);
  CHNS_CUDA(cudaGetLastError());
  return st;
}

chns_status learned_collect(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                            const chns_coef* coef, const double* b, int every, int max_samples,
                            bool with_net, int* added, cudaStream_t s) {
  CHNS_CHECK(L && m && prm && coef && b && added, CHNS_EINVAL, "chns_learned_collect: null argument");
  CHNS_CHECK(every >= 1 && max_samples >= 0, CHNS_EINVAL, "chns_learned_collect: bad sampling");
  *added = 0;
  if (max_samples == 0) return CHNS_OK;
  const int64_t N = m->d.n_nodes;
  double *snaps = nullptr, *xs = nullptr;
  CHNS_CUDA(cudaMallocAsync(&snaps, (size_t)max_samples * N * sizeof(double), s));
  CHNS_CUDA(cudaMallocAsync(&xs, (size_t)N * sizeof(double), s));
  int ns = 0;
  CHNS_CHECK(!with_net || L->out_scale > 0.0, CHNS_EINVAL,
             "chns_learned_collect: the network has no output scale yet (train first)");
  chns_status st = pcg_snapshots(m, prm, coef, b, 1e-10, every, max_samples, snaps, &ns, xs, s,
                                 with_net ? L : nullptr);
  for (int k = 0; k < ns && st == CHNS_OK; ++k) {
    double* e = snaps + (size_t)k * N;
    vec_axpby(1.0, xs, -1.0, e, e, N, s);  // e_k = x* - x_k
    st = learned_add_sample(L, m, prm, coef, e, s);
    if (st == CHNS_OK) ++*added;
  }
  cudaFreeAsync(snaps, s);
  cudaFreeAsync(xs, s);
  CHNS_CUDA(cudaGetLastError());
  return st;
}

}  // namespace chns

// ================================================================== C ABI
extern "C" {

chns_status chns_learned_create(int32_t D, int32_t capacity, uint64_t seed, void* stream,
                                chns_learned** out) {
  using namespace chns::lp;
  CHNS_CHECK(out, CHNS_EINVAL, "chns_learned_create: null out");
  *out = nullptr;
  CHNS_CHECK(D >= 8 && D <= 256 && (D & (D - 1)) == 0, CHNS_EINVAL,
             "chns_learned_create: D must be a power of two in [8, 256]");
  CHNS_CHECK(capacity >= 0, CHNS_EINVAL, "chns_learned_create: negative capacity");
  chns_status st = set_attrs();
  if (st != CHNS_OK) return st;
  cudaStream_t s = as_stream(stream);
  chns_learned* L = new chns_learned();
  L->D = D;
  L->nv = (int64_t)D * D * D;
  L->capacity = capacity;
  L->off = make_offsets();
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&L->sm_count, cudaDevAttrMultiProcessorCount, dev);
  L->wparts = std::min(kMaxParts, 2 * std::max(1, L->sm_count));
  L->oparts = std::min<int>(grid_for(L->nv), 512);
  bool ok = true;
  auto alloc = [&](auto** p, size_t bytes) {
    if (!ok) return;
    if (cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(bytes, 16)) != cudaSuccess) ok = false;
  };
  const size_t np = L->off.total;
  alloc(&L->P, np * 4);
  alloc(&L->G, np * 4);
  alloc(&L->Am, np * 4);
  alloc(&L->Av, np * 4);
  alloc(&L->Wf, kLayers * 27 * 256 * 2);
  alloc(&L->Wt, kLayers * 27 * 256 * 2);
  auto act = [&](int l) { return (size_t)vox(L, l) * kC * 2; };
  alloc(&L->x0, act(0));
  alloc(&L->x2, (size_t)L->nv * 4);
  for (int l = 0; l < 4; ++l) alloc(&L->enc[l], act(l));
  for (int l = 1; l < 4; ++l) alloc(&L->ein[l], act(l));
  for (int l = 0; l < 3; ++l) {
    alloc(&L->din[l], act(l));
    alloc(&L->dec[l], act(l));
    alloc(&L->gdec[l], act(l) * 2);
  }
  for (int l = 1; l < 4; ++l) alloc(&L->gein[l], act(l) * 2);
  alloc(&L->gz, act(0));
  alloc(&L->out, L->nv * 4);
  alloc(&L->wpart, (size_t)L->wparts * kWgOut * 4);
  alloc(&L->opart, (size_t)L->oparts * kOutParts * 4);
  alloc(&L->g_r, L->nv * 4);
  alloc(&L->g_lr, L->nv * 4);
  alloc(&L->g_w, L->nv * 4);
  alloc(&L->g_t, L->nv * 4);
  alloc(&L->dscal, 2048 * 8);
  if (capacity > 0) {
    alloc(&L->rx, (size_t)capacity * L->nv * 4);
    alloc(&L->rt, (size_t)capacity * L->nv * 4);
    L->hs.assign(capacity, 0.0);
    L->heae.assign(capacity, 0.0);
  }
  if (!ok) {
    chns_learned_destroy(L);
    set_error("chns_learned_create: device allocation failed");
    return CHNS_ENOMEM;
  }
  // He-normal conv weights (std sqrt(2 / (27 cin))), zero biases, drawn by a seeded
  // splitmix64 + Box-Muller generator on the host
  std::vector<float> h(np, 0.f);
  uint64_t state = seed;
  auto normal = [&]() {
    const double u1 = ((splitmix64(state) >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = (splitmix64(state) >> 11) * 0x1.0p-53;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
  };
  for (int k = 0; k < kLayers; ++k) {
    const double sd = std::sqrt(2.0 / (27.0 * L->off.cin[k]));
    for (int i = 0; i < 27 * kC * L->off.cin[k]; ++i) h[L->off.w[k] + i] = (float)(sd * normal());
  }
  // the output layer starts at zero: the first correction is c = 0 (energy loss 1), and the
  // gradient reaches the convolutions only once out.W has moved (no early blow-up that would
  // switch all ReLUs off)
  st = chns_learned_set_params(L, h.data());
  if (st != CHNS_OK) {
    chns_learned_destroy(L);
    return st;
  }
  (void)s;
  *out = L;
  return CHNS_OK;
}

void chns_learned_destroy(chns_learned* L) {
  if (!L) return;
  void* ptrs[] = {L->P, L->G, L->Am, L->Av, L->Wf, L->Wt, L->x0, L->x2, L->enc[0], L->enc[1], L->enc[2],
                  L->enc[3], L->ein[1], L->ein[2], L->ein[3], L->din[0], L->din[1], L->din[2],
                  L->dec[0], L->dec[1], L->dec[2], L->gdec[0], L->gdec[1], L->gdec[2],
                  L->gein[1], L->gein[2], L->gein[3], L->gz, L->out, L->wpart, L->opart,
                  L->g_r, L->g_lr, L->g_w, L->g_t, L->dscal, L->rx, L->rt, L->loss_dev,
                  L->re, L->rphi, L->d32, L->w32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete L;
}

int64_t chns_learned_num_params(const chns_learned* L) { return L ? L->off.total : 0; }

chns_status chns_learned_get_params(const chns_learned* L, float* params) {
  CHNS_CHECK(L && params, CHNS_EINVAL, "chns_learned_get_params: null argument");
  CHNS_CUDA(cudaDeviceSynchronize());
  CHNS_CUDA(cudaMemcpy(params, L->P, L->off.total * sizeof(float), cudaMemcpyDeviceToHost));
  return CHNS_OK;
}

chns_status chns_learned_set_params(chns_learned* L, const float* params) {
  CHNS_CHECK(L && params, CHNS_EINVAL, "chns_learned_set_params: null argument");
  CHNS_CUDA(cudaDeviceSynchronize());
  CHNS_CUDA(cudaMemcpy(L->P, params, L->off.total * sizeof(float), cudaMemcpyHostToDevice));
  CHNS_CUDA(cudaMemset(L->Am, 0, L->off.total * sizeof(float)));
  CHNS_CUDA(cudaMemset(L->Av, 0, L->off.total * sizeof(float)));
  L->adam_t = 0;
  chns::lp::pack(L, 0);
  CHNS_CUDA(cudaDeviceSynchronize());
  return CHNS_OK;
}

chns_status chns_learned_set_output_scale(chns_learned* L, double s) {
  CHNS_CHECK(L && s > 0.0 && std::isfinite(s), CHNS_EINVAL, "chns_learned_set_output_scale: bad value");
  L->out_scale = s;
  return CHNS_OK;
}

double chns_learned_output_scale(const chns_learned* L) { return L ? L->out_scale : 0.0; }

chns_status chns_learned_forward(chns_learned* L, const float* x, float* out, void* stream) {
  using namespace chns::lp;
  CHNS_CHECK(L && x && out, CHNS_EINVAL, "chns_learned_forward: null argument");
  cudaStream_t s = as_stream(stream);
  note_launch();
  k_pack_planar<<<grid_for(L->nv), kThreads, 0, s>>>(x, L->x2, L->x0, L->nv);
  chns_status st = forward(L, s);
  if (st != CHNS_OK) return st;
  CHNS_CUDA(cudaMemcpyAsync(out, L->out, L->nv * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return CHNS_OK;
}

chns_status chns_learned_backward(chns_learned* L, const float* gout, float* grad, void* stream) {
  using namespace chns::lp;
  CHNS_CHECK(L && gout && grad, CHNS_EINVAL, "chns_learned_backward: null argument");
  cudaStream_t s = as_stream(stream);
  chns_status st = backward(L, nullptr, 0.f, gout, nullptr, s);
  if (st != CHNS_OK) return st;
  CHNS_CUDA(cudaMemcpyAsync(grad, L->G, L->off.total * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return CHNS_OK;
}

chns_status chns_learned_adam(chns_learned* L, const float* grad, double lr, void* stream) {
  CHNS_CHECK(L && grad && lr > 0.0, CHNS_EINVAL, "chns_learned_adam: bad argument");
  chns::lp::adam(L, grad, lr, as_stream(stream));
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status chns_learned_inputs(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                                const chns_coef* coef, const double* r, float* x, double* s_host,
                                void* stream) {
  using namespace chns::lp;
  CHNS_CHECK(L && m && prm && coef && r && x, CHNS_EINVAL, "chns_learned_inputs: null argument");
  cudaStream_t s = as_stream(stream);
  chns_status st = density_channel(L, m, prm, coef, s);
  if (st != CHNS_OK) return st;
  double rr = 0.0;
  st = dot_host(m, r, r, m->d.n_nodes, &rr, s);
  if (st != CHNS_OK) return st;
  const double sc = std::sqrt(rr / (double)L->nv);
  restrict_to<double>(L, m, r, L->g_r, s);
  // x = (R r / s, density channel) in FP32, before any bfloat16 rounding
  note_launch();
  k_scale_f<<<grid_for(L->nv), kThreads, 0, s>>>(L->g_r, x, L->nv, sc > 0 ? (float)(1.0 / sc) : 0.f);
  CHNS_CUDA(cudaMemcpyAsync(x + L->nv, L->g_lr, L->nv * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (s_host) *s_host = sc;
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status chns_learned_prolong(chns_learned* L, const chns_mesh* m, const float* grid, double* y,
                                 void* stream) {
  using namespace chns::lp;
  CHNS_CHECK(L && m && grid && y, CHNS_EINVAL, "chns_learned_prolong: null argument");
  cudaStream_t s = as_stream(stream);
  const int64_t N = m->d.n_nodes;
  note_launch();
  k_prolong<double><<<grid_for(N), kThreads, 0, s>>>(grid, m->d_node_int, N, L->D,
                                                     grid_scale(L->D), nullptr, 0.f, 1.f, nullptr,
                                                     nullptr, y);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status chns_learned_add_sample(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                                    const chns_coef* coef, const double* e, void* stream) {
  return chns::learned_add_sample(L, m, prm, coef, e, as_stream(stream));
}

chns_status chns_learned_collect(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                                 const chns_coef* coef, const double* b, int32_t every,
                                 int32_t max_samples, int32_t with_net, int32_t* added,
                                 void* stream) {
  int a = 0;
  chns_status st = chns::learned_collect(L, m, prm, coef, b, every, max_samples, with_net != 0, &a,
                                         as_stream(stream));
  if (added) *added = a;
  return st;
}

int32_t chns_learned_num_samples(const chns_learned* L) { return L ? L->count : 0; }

chns_status chns_learned_train(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                               int32_t iterations, double lr, uint64_t seed, float* loss_host,
                               void* stream) {
  using namespace chns::lp;
  CHNS_CHECK(L && m && prm && iterations >= 0 && lr > 0.0, CHNS_EINVAL,
             "chns_learned_train: bad argument");
  CHNS_CHECK(L->count > 0, CHNS_EINVAL, "chns_learned_train: the replay buffer is empty");
  CHNS_CHECK(L->bound == m, CHNS_EINVAL, "chns_learned_train: the pairs belong to another mesh");
  cudaStream_t s = as_stream(stream);
  if (L->out_scale <= 0.0) {
    double tot = 0.0;
    for (int k = 0; k < L->count; ++k) {
      double q = 0.0;
      chns_status st = grid_sq(L, L->rt + (size_t)k * L->nv, &q, s);
      if (st != CHNS_OK) return st;
      tot += q;
    }
    const double rms = std::sqrt(tot / ((double)L->count * (double)L->nv));
    L->out_scale = rms > 0.0 && std::isfinite(rms) ? rms : 1.0;
  }
  if (L->loss_cap < iterations) {
    if (L->loss_dev) cudaFree(L->loss_dev);
    L->loss_dev = nullptr;
    CHNS_CUDA(cudaMalloc(&L->loss_dev, std::max(iterations, 1) * sizeof(float)));
    L->loss_cap = iterations;
  }
  if (iterations > 0)
    CHNS_CUDA(cudaMemsetAsync(L->loss_dev, 0, iterations * sizeof(float), s));
  const int64_t N = L->bound_n;
  const unsigned nb = std::min<unsigned>(grid_for(N), 1024);
  uint64_t st_rng = seed;
  for (int it = 0; it < iterations; ++it) {
    const int k = (int)(splitmix64(st_rng) % (uint64_t)L->count);
    const double sc = L->hs[k] * L->out_scale, eae = L->heae[k];
    if (!(eae > 0.0) || !std::isfinite(eae)) continue;
    note_launch();
    k_load_pair<<<grid_for(L->nv), kThreads, 0, s>>>(L->rx + (size_t)k * L->nv, L->x2, L->x0,
                                                     L->nv);
    chns_status st = forward(L, s);
    if (st != CHNS_OK) return st;
    // d = e - c, w = A d with the pair's coefficients (FP32 apply, bfloat16 coefficient)
    note_launch();
    k_prolong_diff<<<grid_for(N), kThreads, 0, s>>>(L->out, m->d_node_int, N, L->D,
                                                    grid_scale(L->D), (float)sc,
                                                    L->re + (size_t)k * N, L->d32);
    chns_coef ck{};
    ck.phi_tilde = L->rphi + (size_t)k * N;
    st = apply_op(m, CHNS_OP_POISSON, prm, &ck, L->d32, L->w32, CHNS_FP32_BF16COEF, s);
    if (st != CHNS_OK) return st;
    note_launch();
    k_dot_acc<<<nb, kThreads, 0, s>>>(L->d32, L->w32, N, (float)(1.0 / eae), L->loss_dev + it);
    // dL/d(out) = -2 sc P_g^T (A d) / e^T A e, divided by the loss where it exceeds 1
    restrict_to<float>(L, m, L->w32, L->g_t, s);
    note_launch();
    k_scale_grad<<<grid_for(L->nv), kThreads, 0, s>>>(L->g_t, L->g_r, L->nv,
                                                      (float)(-2.0 * sc / eae), L->loss_dev + it);
    st = backward(L, nullptr, 0.f, L->g_r, nullptr, s);
    if (st != CHNS_OK) return st;
    adam(L, L->G, lr, s);
  }
  CHNS_CUDA(cudaGetLastError());
  if (loss_host && iterations > 0) {
    CHNS_CUDA(cudaMemcpyAsync(loss_host, L->loss_dev, iterations * sizeof(float),
                              cudaMemcpyDeviceToHost, s));
    CHNS_CUDA(cudaStreamSynchronize(s));
  }
  return CHNS_OK;
}

}  // extern "C"
