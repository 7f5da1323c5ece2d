// Learned warm start: a 3D convolutional U-Net that predicts the Newton
// update from the residual, ln k, s_w and the previous update, trained on
// systems the simulator solves.  Not part of the paper's method.
//
// Architecture (4 resolution levels, 32 channels, 3x3x3 kernels):
//   c00,c01 | pool | c10,c11 | pool | c20,c21 | pool | c30,c31
//   up, concat [up, skip] -> d20,d21 | up, concat -> d10,d11 | up, concat -> d00,d01 | head h
// conv: Z[v,o] = b[o] + sum_{d in {-1,0,1}^3} sum_c X[v+d, c] W[t(d), o, c]
// (X = 0 outside the grid, t(d) = (dx+1) + 3(dy+1) + 9(dz+1)), ReLU after
// every conv but the head; pool: average of the existing children (coarse
// size ceil(n/2)); up: nearest parent.  Loss 0.5/n sum (Y - T)^2 over the two
// predicted channels.
//
// Data layout: activations are BF16, voxel-major with the channels
// contiguous ([v][C], v = i + nx (j + ny k), the simulator's cell order).
// The network input has 16 channels (8 used; the rest stay zero so every
// contraction is a whole number of 16-wide MMA steps).  Weights: FP32 master
// copy [27][Co][Ci] (+ Adam moments), and two BF16 copies made after every
// update: [27][Co][Ci] for the forward pass and the tap-flipped transpose
// [26-t][Ci][Co] for the data gradient, which is then the same kernel.
//
// Every contraction runs on the tensor cores: mma.sync m16n8k16 BF16 with
// FP32 accumulation.  The forward/data-gradient kernel is an implicit GEMM
// (M = voxels, N = output channels, K = 27 taps x input channels): each tap's
// shifted input rows and weight slice are staged in shared memory with
// cp.async (zero-fill outside the grid), double buffered across taps, and
// fed to the MMAs with ldmatrix.  The weight-gradient kernel contracts over
// voxels (M = output channels, N = input channels) with ldmatrix.trans from
// the voxel-major tiles, one CTA per (voxel chunk, tap), partials reduced in
// a fixed order so results do not depend on scheduling.
#include "common.cuh"
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <memory>
#include <mutex>

typedef __nv_bfloat16 bf16;

namespace nn {

constexpr int NLAYER = 15;
constexpr int CIN_GPU = 16;     // channels of the input feature tensor on the device
constexpr int CIN_USED = 8;     // the network's input channels
constexpr int COUT_HEAD = 8;    // head outputs (the first two are the prediction)
constexpr int NPRED = 2;

struct layer_def { const char *name; int ci, co, relu; };
// ci is the device-side input width (the input layer is padded from 8 to 16)
static const layer_def LAYERS[NLAYER] = {
    {"c00", 16, 32, 1}, {"c01", 32, 32, 1}, {"c10", 32, 32, 1}, {"c11", 32, 32, 1},
    {"c20", 32, 32, 1}, {"c21", 32, 32, 1}, {"c30", 32, 32, 1}, {"c31", 32, 32, 1},
    {"d20", 64, 32, 1}, {"d21", 32, 32, 1}, {"d10", 64, 32, 1}, {"d11", 32, 32, 1},
    {"d00", 64, 32, 1}, {"d01", 32, 32, 1}, {"h", 32, 8, 0}};
enum { C00, C01, C10, C11, C20, C21, C30, C31, D20, D21, D10, D11, D00, D01, HEAD };

static inline int ci_true(int l) { return l == C00 ? CIN_USED : LAYERS[l].ci; }
static inline int cob(int l) { return std::max(16, LAYERS[l].co); }   // data-gradient input width

// ------------------------------------------------------------ PTX helpers -
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }
__device__ __forceinline__ void ldsm_x4(unsigned r[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(unsigned r[2], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned r[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// --------------------------------------------------- implicit-GEMM conv ---
// out[v, o] for v in this CTA's 128 voxels, o < NT*8.
// MODE 0: BF16 out = act(acc + bias)           (forward)
// MODE 1: FP32 out = acc + bias                (head forward)
// MODE 2: BF16 out = acc * (mask[v, o] > 0)    (data gradient through a ReLU)
// MODE 3: BF16 out = acc                       (data gradient, no ReLU below)
constexpr int CBM = 128;    // voxels per CTA (4 warps x 32)
template <int CI, int NT>
struct conv_smem {
  static constexpr int AST = CI + 8, BST = CI + 8, CO = NT * 8;
  static constexpr int A_EL = CBM * AST, B_EL = CO * BST;
  static constexpr int BYTES = 2 * (A_EL + B_EL) * 2;
};

template <int CI, int NT, int MODE>
__global__ void __launch_bounds__(128) k_conv(int nx, int ny, int nz, const bf16 *__restrict__ X, int ldx, int offx,
                                              const bf16 *__restrict__ Wt, const float *__restrict__ bias, int relu,
                                              void *out, int ldo, int offo, const bf16 *__restrict__ mask, int ldm,
                                              int offm) {
  typedef conv_smem<CI, NT> S;
  constexpr int CO = NT * 8, CH = CI / 8;            // 16-byte chunks per input row
  constexpr int AJ = CBM * CH / 128;                  // A chunks per thread and tap
  constexpr int BJ = (CO * CH + 127) / 128;           // B chunks per thread and tap
  extern __shared__ __align__(16) unsigned char smraw[];
  bf16 *sA = reinterpret_cast<bf16 *>(smraw);
  bf16 *sB = sA + 2 * S::A_EL;
  const int V = nx * ny * nz, nxy = nx * ny;
  const int v0 = blockIdx.x * CBM, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // the voxels whose input rows this thread copies (same for every tap)
  int vx[AJ], vy[AJ], vz[AJ], vrow[AJ], vch[AJ];
#pragma unroll
  for (int j = 0; j < AJ; j++) {
    int q = j * 128 + t;
    vrow[j] = q / CH; vch[j] = q % CH;
    int v = v0 + vrow[j];
    if (v < V) { vz[j] = v / nxy; int r = v - vz[j] * nxy; vy[j] = r / nx; vx[j] = r - vy[j] * nx; }
    else { vx[j] = -1000000; vy[j] = 0; vz[j] = 0; }
  }
  auto load = [&](int stage, int tap) {
    int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
    bf16 *a = sA + stage * S::A_EL;
#pragma unroll
    for (int j = 0; j < AJ; j++) {
      int x = vx[j] + dx, y = vy[j] + dy, z = vz[j] + dz;
      bool ok = x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz;
      const bf16 *src = ok ? X + ((size_t)(x + nx * (y + ny * z)) * ldx + offx + vch[j] * 8) : X;
      cp_async16(a + vrow[j] * S::AST + vch[j] * 8, src, ok ? 16 : 0);
    }
    bf16 *b = sB + stage * S::B_EL;
    const bf16 *w = Wt + (size_t)tap * CO * CI;
#pragma unroll
    for (int j = 0; j < BJ; j++) {
      int q = j * 128 + t;
      if (q < CO * CH) {
        int o = q / CH, ch = q % CH;
        cp_async16(b + o * S::BST + ch * 8, w + o * CI + ch * 8, 16);
      }
    }
  };
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int nt = 0; nt < NT; nt++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[mt][nt][e] = 0.f;

  load(0, 0);
  cp_commit();
  for (int tap = 0; tap < 27; tap++) {
    if (tap + 1 < 27) { load((tap + 1) & 1, tap + 1); cp_commit(); cp_wait<1>(); }
    else cp_wait<0>();
    __syncthreads();
    const bf16 *a = sA + (tap & 1) * S::A_EL;
    const bf16 *b = sB + (tap & 1) * S::B_EL;
#pragma unroll
    for (int ks = 0; ks < CI / 16; ks++) {
      unsigned af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; mt++)
        ldsm_x4(af[mt], a + (warp * 32 + mt * 16 + (lane & 15)) * S::AST + ks * 16 + (lane >> 4) * 8);
      unsigned bfr[NT][2];
      if constexpr (NT == 1) {
        ldsm_x2(bfr[0], b + (lane & 7) * S::BST + ks * 16 + ((lane >> 3) & 1) * 8);
      } else {
#pragma unroll
        for (int np = 0; np < NT / 2; np++) {
          unsigned r[4];
          ldsm_x4(r, b + (np * 16 + (lane & 7) + ((lane >> 4) << 3)) * S::BST + ks * 16 + ((lane >> 3) & 1) * 8);
          bfr[2 * np][0] = r[0]; bfr[2 * np][1] = r[1];
          bfr[2 * np + 1][0] = r[2]; bfr[2 * np + 1][1] = r[3];
        }
      }
#pragma unroll
      for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++) mma16816(acc[mt][nt], af[mt], bfr[nt]);
    }
    __syncthreads();                                  // the stage is reloaded two taps later
  }
  // epilogue
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int hh = 0; hh < 2; hh++) {
      int v = v0 + warp * 32 + mt * 16 + (lane >> 2) + hh * 8;
      if (v >= V) continue;
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        int o = nt * 8 + (lane & 3) * 2;
        float y0 = acc[mt][nt][2 * hh], y1 = acc[mt][nt][2 * hh + 1];
        if (MODE == 0 || MODE == 1) { y0 += bias[o]; y1 += bias[o + 1]; }
        if (MODE == 0 && relu) { y0 = fmaxf(y0, 0.f); y1 = fmaxf(y1, 0.f); }
        if (MODE == 2) {
          __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(mask + (size_t)v * ldm + offm + o);
          if (!(__bfloat162float(m.x) > 0.f)) y0 = 0.f;
          if (!(__bfloat162float(m.y) > 0.f)) y1 = 0.f;
        }
        if (MODE == 1) {
          float *op = reinterpret_cast<float *>(out) + (size_t)v * ldo + offo + o;
          op[0] = y0; op[1] = y1;
        } else {
          *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(out) + (size_t)v * ldo + offo + o) =
              __floats2bfloat162_rn(y0, y1);
        }
      }
    }
}

// ------------------------------------------- halo-tiled forward conv ------
// The forward contraction (MODE 0 / 1 of k_conv) with the input read once per
// tile: a CTA owns an 8 x 4 x 4 box of output voxels (row r = x + 8 y + 32 z,
// warp w = z-slice w), stages the 10 x 6 x 6 input halo in shared memory
// (cp.async, zero-filled outside the grid) and, for each of the 27 taps,
// reads its A fragments straight from the halo with per-lane ldmatrix row
// addresses (the shifted voxel of each output row), so only the tap's
// weights stream per tap (two stages).  k_conv gathers 128 shifted rows per
// tap instead, 27 reads of the input per tile.  MMAs are issued in the same
// tap / K order as k_conv.
constexpr int HX = 8, HY = 4, HZ = 4;                         // output box
constexpr int HHX = HX + 2, HHY = HY + 2, HHZ = HZ + 2, HNV = HHX * HHY * HHZ;
template <int CI, int NT>
struct halo_smem {
  static constexpr int AST = CI + 8, BST = CI + 8, CO = NT * 8;
  static constexpr int A_EL = HNV * AST, B_EL = CO * BST;
  static constexpr int BYTES = (A_EL + 2 * B_EL) * 2;
};
template <int CI, int NT, int MODE>
__global__ void __launch_bounds__(128) k_conv_halo(int nx, int ny, int nz, const bf16 *__restrict__ X, int ldx,
                                                   int offx, const bf16 *__restrict__ Wt,
                                                   const float *__restrict__ bias, int relu, void *out, int ldo,
                                                   int offo) {
  typedef halo_smem<CI, NT> S;
  constexpr int CO = NT * 8, CH = CI / 8;
  constexpr int BJ = (CO * CH + 127) / 128;
  extern __shared__ __align__(16) unsigned char smraw[];
  bf16 *sA = reinterpret_cast<bf16 *>(smraw);
  bf16 *sB = sA + S::A_EL;
  const int tx = (nx + HX - 1) / HX, ty = (ny + HY - 1) / HY;
  const int bx = blockIdx.x % tx, by = (blockIdx.x / tx) % ty, bz = blockIdx.x / (tx * ty);
  const int X0 = bx * HX, Y0 = by * HY, Z0 = bz * HZ;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // the halo: HNV voxels x CH chunks of 16 bytes
  for (int q = t; q < HNV * CH; q += 128) {
    int h = q / CH, ch = q % CH;
    int hx = h % HHX, hy = (h / HHX) % HHY, hz = h / (HHX * HHY);
    int x = X0 + hx - 1, y = Y0 + hy - 1, z = Z0 + hz - 1;
    bool ok = x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz;
    const bf16 *src = ok ? X + ((size_t)(x + nx * (y + ny * z)) * ldx + offx + ch * 8) : X;
    cp_async16(sA + h * S::AST + ch * 8, src, ok ? 16 : 0);
  }
  auto loadw = [&](int stage, int tap) {
    bf16 *b = sB + stage * S::B_EL;
    const bf16 *w = Wt + (size_t)tap * CO * CI;
#pragma unroll
    for (int j = 0; j < BJ; j++) {
      int q = j * 128 + t;
      if (q < CO * CH) {
        int o = q / CH, ch = q % CH;
        cp_async16(b + o * S::BST + ch * 8, w + o * CI + ch * 8, 16);
      }
    }
  };
  loadw(0, 0);
  cp_commit();
  // halo row of output row (warp, mt, lane & 15) at the centre tap
  int hbase[2];
#pragma unroll
  for (int mt = 0; mt < 2; mt++) {
    int r = warp * 32 + mt * 16 + (lane & 15);
    int x = r % HX, y = (r / HX) % HY, z = r / (HX * HY);
    hbase[mt] = (x + 1) + HHX * ((y + 1) + HHY * (z + 1));
  }
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int nt = 0; nt < NT; nt++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[mt][nt][e] = 0.f;
  for (int tap = 0; tap < 27; tap++) {
    if (tap + 1 < 27) { loadw((tap + 1) & 1, tap + 1); cp_commit(); cp_wait<1>(); }
    else cp_wait<0>();
    __syncthreads();
    const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
    const int shift = dx + HHX * (dy + HHY * dz);
    const bf16 *b = sB + (tap & 1) * S::B_EL;
#pragma unroll
    for (int ks = 0; ks < CI / 16; ks++) {
      unsigned af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; mt++)
        ldsm_x4(af[mt], sA + (hbase[mt] + shift) * S::AST + ks * 16 + (lane >> 4) * 8);
      unsigned bfr[NT][2];
      if constexpr (NT == 1) {
        ldsm_x2(bfr[0], b + (lane & 7) * S::BST + ks * 16 + ((lane >> 3) & 1) * 8);
      } else {
#pragma unroll
        for (int np = 0; np < NT / 2; np++) {
          unsigned r[4];
          ldsm_x4(r, b + (np * 16 + (lane & 7) + ((lane >> 4) << 3)) * S::BST + ks * 16 + ((lane >> 3) & 1) * 8);
          bfr[2 * np][0] = r[0]; bfr[2 * np][1] = r[1];
          bfr[2 * np + 1][0] = r[2]; bfr[2 * np + 1][1] = r[3];
        }
      }
#pragma unroll
      for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++) mma16816(acc[mt][nt], af[mt], bfr[nt]);
    }
    __syncthreads();                                  // the weight stage is reloaded two taps later
  }
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int hh = 0; hh < 2; hh++) {
      int r = warp * 32 + mt * 16 + (lane >> 2) + hh * 8;
      int x = X0 + r % HX, y = Y0 + (r / HX) % HY, z = Z0 + r / (HX * HY);
      if (x >= nx || y >= ny || z >= nz) continue;
      size_t v = (size_t)x + (size_t)nx * (y + (size_t)ny * z);
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        int o = nt * 8 + (lane & 3) * 2;
        float y0 = acc[mt][nt][2 * hh] + bias[o], y1 = acc[mt][nt][2 * hh + 1] + bias[o + 1];
        if (MODE == 0 && relu) { y0 = fmaxf(y0, 0.f); y1 = fmaxf(y1, 0.f); }
        if (MODE == 1) {
          float *op = reinterpret_cast<float *>(out) + v * ldo + offo + o;
          op[0] = y0; op[1] = y1;
        } else {
          *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(out) + v * ldo + offo + o) =
              __floats2bfloat162_rn(y0, y1);
        }
      }
    }
}

// ------------------------------------------ implicit-GEMM conv, tcgen05 ---
// The same contraction on the 5th-generation tensor cores: per CTA a tile of
// 128 voxels (M) against CO output channels (N = 32 or 64), K = 27 taps x CI.
// For every tap the CTA gathers the 128 shifted input rows (cp.async,
// zero-filled outside the grid) and the tap's CO x CI weights into shared
// memory in the K-major, no-swizzle core-matrix layout (8 rows x 16 bytes per
// 128-byte core matrix; the two 8-element halves of a 16-wide K block 128 B
// apart, 8-row groups 256 B apart), then one thread issues CI/16
// tcgen05.mma.kind::f16 (BF16 x BF16 -> FP32) into a TMEM accumulator of
// 128 lanes x CO columns.  Two stages: a stage is refilled once the MMAs that
// read it have committed to that stage's mbarrier.  The epilogue reads the
// accumulator with tcgen05.ld (thread = voxel row) and applies bias / ReLU or
// the data-gradient mask.  Every wait is bounded; on a timeout the kernel
// records an error and writes nothing.
__device__ __forceinline__ uint64_t tc_desc(unsigned saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;             // leading byte offset: the K halves of a block
  d |= (uint64_t)(256 >> 4) << 32;             // stride byte offset: consecutive 8-row groups
  d |= (uint64_t)1 << 46;                      // descriptor version; no swizzle, base offset 0
  return d;
}
__device__ __forceinline__ uint32_t tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ bool tc_wait(uint64_t *bar, unsigned parity) {
  for (int it = 0; it < (1 << 24); it++) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                 "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                 "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 32; c++) v[c] = __uint_as_float(r[c]);
}

template <int CI, int CO>
struct tc_smem {
  static constexpr int KB = CI / 16;
  static constexpr int A_BYTES = KB * (CBM / 8) * 256, B_BYTES = KB * (CO / 8) * 256;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int NS = 4;                   // stages: 2 taps of copies ahead + 2 of MMA slack
  static constexpr int BYTES = NS * STAGE;
};

// MODE as for k_conv: 0 forward (bias, ReLU flag), 2 data gradient with mask,
// 3 data gradient.  Persistent: each CTA walks tiles blockIdx.x, +gridDim.x, ...
// with one TMEM allocation; taps flow through NS shared-memory stages, a
// stage being refilled once the MMAs that read it have committed.
template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(128) k_conv_tc(int nx, int ny, int nz, const bf16 *__restrict__ X, int ldx, int offx,
                                                 const bf16 *__restrict__ Wt, const float *__restrict__ bias, int relu,
                                                 bf16 *out, int ldo, int offo, const bf16 *__restrict__ mask, int ldm,
                                                 int offm, int *err) {
  typedef tc_smem<CI, CO> S;
  constexpr int CH = CI / 8, AJ = CBM * CH / 128, BJ = (CO * CH + 127) / 128, NS = S::NS;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ uint64_t bar[NS];
  __shared__ uint32_t tslot;
  const int V = nx * ny * nz, nxy = nx * ny, ntile = (V + CBM - 1) / CBM;
  const int t = threadIdx.x, warp = t >> 5;
  auto coff = [](int r, int ch) { return (r >> 3) * 256 + (ch & 1) * 128 + (r & 7) * 16; };
  if (t == 0) {
    for (int k = 0; k < NS; k++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[k])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)), "n"(CO) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tslot, idesc = tc_idesc(CO);
  bool ok = true;
  long long g0 = 0;                               // taps issued by this CTA before the current tile
  for (int tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x, g0 += 27) {
    const int v0 = tile * CBM;
    int vx[AJ], vy[AJ], vz[AJ], vrow[AJ], vch[AJ];
#pragma unroll
    for (int j = 0; j < AJ; j++) {
      int q = j * 128 + t;
      vrow[j] = q / CH; vch[j] = q % CH;
      int v = v0 + vrow[j];
      if (v < V) { vz[j] = v / nxy; int r = v - vz[j] * nxy; vy[j] = r / nx; vx[j] = r - vy[j] * nx; }
      else { vx[j] = -1000000; vy[j] = 0; vz[j] = 0; }
    }
    // tap u of this tile is global tap g0 + u: stage (g0 + u) % NS, and its
    // commit is completion number (g0 + u) / NS of that stage's barrier
    auto load = [&](int u) {
      long long g = g0 + u;
      int stage = (int)(g % NS);
      if (g >= NS) ok = ok && tc_wait(&bar[stage], (unsigned)(((g - NS) / NS) & 1));   // MMAs of g - NS done
      int dx = u % 3 - 1, dy = (u / 3) % 3 - 1, dz = u / 9 - 1;
      unsigned char *a = smraw + stage * S::STAGE, *b = a + S::A_BYTES;
#pragma unroll
      for (int j = 0; j < AJ; j++) {
        int x = vx[j] + dx, y = vy[j] + dy, z = vz[j] + dz;
        bool in = x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz;
        const bf16 *src = in ? X + ((size_t)(x + nx * (y + ny * z)) * ldx + offx + vch[j] * 8) : X;
        cp_async16(a + (vch[j] >> 1) * (CBM / 8) * 256 + coff(vrow[j], vch[j]), src, in ? 16 : 0);
      }
      const bf16 *w = Wt + (size_t)u * CO * CI;
#pragma unroll
      for (int j = 0; j < BJ; j++) {
        int q = j * 128 + t;
        if (q < CO * CH) {
          int o = q / CH, ch = q % CH;
          cp_async16(b + (ch >> 1) * (CO / 8) * 256 + coff(o, ch), w + o * CI + ch * 8, 16);
        }
      }
    };
    // copies run LA = NS - 2 taps ahead, so the stage refilled at tap t was
    // last read by the MMAs of tap t - 2, which have had a whole tap to finish
    constexpr int LA = NS - 2;
#pragma unroll 1
    for (int u = 0; u < LA; u++) { load(u); cp_commit(); }
    for (int tap = 0; tap < 27; tap++) {
      int u = tap + LA;
      if (u < 27) load(u);
      cp_commit();                                // (possibly empty) group: one per tap
      cp_wait<LA>();                              // this tap's copies have landed
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ok = __syncthreads_and(ok);
      if (t == 0 && ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        long long g = g0 + tap;
        int stage = (int)(g % NS);
        unsigned char *a = smraw + stage * S::STAGE, *b = a + S::A_BYTES;
#pragma unroll
        for (int kb = 0; kb < S::KB; kb++) {
          uint64_t da = tc_desc(smem_u32(a + kb * (CBM / 8) * 256)), db = tc_desc(smem_u32(b + kb * (CO / 8) * 256));
          uint32_t acc = (tap > 0 || kb > 0) ? 1u : 0u;
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                       ::"r"(taddr), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&bar[stage])) : "memory");
      }
    }
    // the tile's last MMAs have committed
    {
      long long g = g0 + 26;
      ok = ok && tc_wait(&bar[(int)(g % NS)], (unsigned)((g / NS) & 1));
    }
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      int v = v0 + t;                             // TMEM lane = row = thread
#pragma unroll
      for (int c0 = 0; c0 < CO; c0 += 32) {
        float acc[32];
        tc_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
        if (v < V) {
          if (MODE == 0) {
#pragma unroll
            for (int c = 0; c < 32; c++) { acc[c] += bias[c0 + c]; if (relu) acc[c] = fmaxf(acc[c], 0.f); }
          } else if (MODE == 2) {
            const bf16 *mk = mask + (size_t)v * ldm + offm + c0;
#pragma unroll
            for (int c = 0; c < 32; c++) if (!(__bfloat162float(mk[c]) > 0.f)) acc[c] = 0.f;
          }
          uint4 pk[4];
          __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(pk);
#pragma unroll
          for (int c = 0; c < 16; c++) h2[c] = __floats2bfloat162_rn(acc[2 * c], acc[2 * c + 1]);
          uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)v * ldo + offo + c0);
#pragma unroll
          for (int u = 0; u < 4; u++) dst[u] = pk[u];
        }
      }
    }
    // the accumulator is read before the next tile's first MMA overwrites it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok && t == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(CO) : "memory");
}

// ------------------------------------------------------ weight gradient ---
// part[tap][chunk][o][c] = sum over the chunk's voxels v of dZ[v, o] X[v + d(tap), c]
// (o < CO, c < CI), and for the centre tap bpart[chunk][o] = sum_v dZ[v, o].
constexpr int WCH = 256;      // voxels per sub-chunk (8 warps x 32)
constexpr int WIT = 4;        // sub-chunks per CTA
template <int CI, int MT>
struct wg_smem {
  static constexpr int ZST = MT * 16 + 8, XST = CI + 8;
  static constexpr int Z_EL = WCH * ZST, X_EL = WCH * XST;
  static constexpr int RED = 8 * MT * 16 * CI;           // floats
  static constexpr int BYTES = (Z_EL + X_EL) * 2 + RED * 4;
};

template <int CI, int MT>
__global__ void __launch_bounds__(256) k_conv_wgrad(int nx, int ny, int nz, const bf16 *__restrict__ X, int ldx,
                                                    int offx, const bf16 *__restrict__ dZ, int ldz, int offz, int co,
                                                    float *part, float *bpart) {
  typedef wg_smem<CI, MT> S;
  constexpr int M16 = MT * 16, CH = CI / 8, NTL = CI / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  bf16 *sZ = reinterpret_cast<bf16 *>(smraw);
  bf16 *sX = sZ + S::Z_EL;
  float *red = reinterpret_cast<float *>(sX + S::X_EL);
  const int V = nx * ny * nz, nxy = nx * ny;
  const int chunk = blockIdx.x, tap = blockIdx.y, nchunk = gridDim.x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
  float acc[MT][NTL][4];
#pragma unroll
  for (int mt = 0; mt < MT; mt++)
#pragma unroll
    for (int nt = 0; nt < NTL; nt++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[mt][nt][e] = 0.f;
  float bsum = 0.f;
  for (int it = 0; it < WIT; it++) {
    int vb = (chunk * WIT + it) * WCH;
    if (vb >= V) break;
    // dZ rows (zero past the end and in the padding channels)
    for (int q = t; q < WCH * (M16 / 8); q += 256) {
      int r = q / (M16 / 8), ch = q % (M16 / 8), v = vb + r;
      bool ok = v < V && ch * 8 < co;
      cp_async16(sZ + r * S::ZST + ch * 8, ok ? dZ + (size_t)v * ldz + offz + ch * 8 : dZ, ok ? 16 : 0);
    }
    // shifted X rows
    for (int q = t; q < WCH * CH; q += 256) {
      int r = q / CH, ch = q % CH, v = vb + r;
      bool ok = false;
      const bf16 *src = X;
      if (v < V) {
        int z = v / nxy, rr = v - z * nxy, y = rr / nx, x = rr - y * nx;
        x += dx; y += dy; z += dz;
        ok = x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz;
        if (ok) src = X + (size_t)(x + nx * (y + ny * z)) * ldx + offx + ch * 8;
      }
      cp_async16(sX + r * S::XST + ch * 8, src, ok ? 16 : 0);
    }
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    if (tap == 13 && t < co)
      for (int r = 0; r < WCH; r++) bsum += __bfloat162float(sZ[r * S::ZST + t]);
#pragma unroll
    for (int ks = 0; ks < 2; ks++) {
      int kb = warp * 32 + ks * 16;
      unsigned af[MT][4];
#pragma unroll
      for (int mt = 0; mt < MT; mt++)
        ldsm_x4_t(af[mt], sZ + (kb + (lane & 7) + ((lane >> 4) << 3)) * S::ZST + mt * 16 + ((lane >> 3) & 1) * 8);
#pragma unroll
      for (int np = 0; np < NTL / 2; np++) {
        unsigned r[4];
        ldsm_x4_t(r, sX + (kb + (lane & 7) + (((lane >> 3) & 1) << 3)) * S::XST + np * 16 + (lane >> 4) * 8);
        unsigned b0[2] = {r[0], r[1]}, b1[2] = {r[2], r[3]};
#pragma unroll
        for (int mt = 0; mt < MT; mt++) {
          mma16816(acc[mt][2 * np], af[mt], b0);
          mma16816(acc[mt][2 * np + 1], af[mt], b1);
        }
      }
    }
    __syncthreads();
  }
  // cross-warp sum in a fixed order
#pragma unroll
  for (int mt = 0; mt < MT; mt++)
#pragma unroll
    for (int nt = 0; nt < NTL; nt++)
#pragma unroll
      for (int e = 0; e < 4; e++) {
        int m = mt * 16 + (lane >> 2) + (e >> 1) * 8, n = nt * 8 + (lane & 3) * 2 + (e & 1);
        red[(warp * M16 + m) * CI + n] = acc[mt][nt][e];
      }
  __syncthreads();
  float *dst = part + ((size_t)tap * nchunk + chunk) * co * CI;
  for (int q = t; q < co * CI; q += 256) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < 8; w++) s += red[w * M16 * CI + q];
    dst[q] = s;
  }
  if (tap == 13 && t < co) bpart[(size_t)chunk * co + t] = bsum;
}

// grad[tap][o][c] += sum over chunks (in order) of part[tap][chunk][o][c]; bias likewise
__global__ void k_wgrad_reduce(int nchunk, int per_tap, const float *part, const float *bpart, int co, float *gW,
                               float *gb) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 27 * per_tap) {
    int tap = q / per_tap, e = q - tap * per_tap;
    const float *p = part + (size_t)tap * nchunk * per_tap + e;
    float s = 0.f;
    for (int c = 0; c < nchunk; c++) s += p[(size_t)c * per_tap];
    gW[q] += s;
  } else if (q < 27 * per_tap + co) {
    int o = q - 27 * per_tap;
    float s = 0.f;
    for (int c = 0; c < nchunk; c++) s += bpart[(size_t)c * co + o];
    gb[o] += s;
  }
}

// ------------------------------------------------------- pool and up ------
struct dims { int nx, ny, nz; __host__ __device__ int V() const { return nx * ny * nz; } };
__host__ __device__ inline dims coarse(dims d) { return {(d.nx + 1) / 2, (d.ny + 1) / 2, (d.nz + 1) / 2}; }

// P[V, c] = mean of the existing children, 32 channels, 8 per thread
__global__ void k_pool(dims f, dims c, const bf16 *X, int ldx, int offx, bf16 *P) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= c.V() * 4) return;
  int V = q >> 2, g = (q & 3) * 8;
  int Z = V / (c.nx * c.ny), r = V - Z * c.nx * c.ny, Y = r / c.nx, Xc = r - Y * c.nx;
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int cnt = 0;
  for (int k = 0; k < 2; k++)
    for (int j = 0; j < 2; j++)
      for (int i = 0; i < 2; i++) {
        int x = 2 * Xc + i, y = 2 * Y + j, z = 2 * Z + k;
        if (x >= f.nx || y >= f.ny || z >= f.nz) continue;
        const bf16 *p = X + (size_t)(x + f.nx * (y + f.ny * z)) * ldx + offx + g;
        uint4 u = *reinterpret_cast<const uint4 *>(p);
        const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
        for (int a = 0; a < 8; a++) s[a] += __bfloat162float(e[a]);
        cnt++;
      }
  uint4 o;
  bf16 *e = reinterpret_cast<bf16 *>(&o);
#pragma unroll
  for (int a = 0; a < 8; a++) e[a] = __float2bfloat16_rn(s[a] / (float)cnt);
  *reinterpret_cast<uint4 *>(P + (size_t)V * 32 + g) = o;
}

// out[v, off + c] = C[parent(v), c], 32 channels
__global__ void k_up(dims f, dims c, const bf16 *C, bf16 *out, int ldo, int offo) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= f.V() * 4) return;
  int v = q >> 2, g = (q & 3) * 8;
  int z = v / (f.nx * f.ny), r = v - z * f.nx * f.ny, y = r / f.nx, x = r - y * f.nx;
  int P = (x >> 1) + c.nx * ((y >> 1) + c.ny * (z >> 1));
  *reinterpret_cast<uint4 *>(out + (size_t)v * ldo + offo + g) = *reinterpret_cast<const uint4 *>(C + (size_t)P * 32 + g);
}

// dC[V, c] = sum over children of G[v, offg + c]  (32 channels)
__global__ void k_up_back(dims f, dims c, const bf16 *G, int ldg, int offg, bf16 *dC) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= c.V() * 4) return;
  int V = q >> 2, g = (q & 3) * 8;
  int Z = V / (c.nx * c.ny), r = V - Z * c.nx * c.ny, Y = r / c.nx, Xc = r - Y * c.nx;
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < 2; k++)
    for (int j = 0; j < 2; j++)
      for (int i = 0; i < 2; i++) {
        int x = 2 * Xc + i, y = 2 * Y + j, z = 2 * Z + k;
        if (x >= f.nx || y >= f.ny || z >= f.nz) continue;
        uint4 u = *reinterpret_cast<const uint4 *>(G + (size_t)(x + f.nx * (y + f.ny * z)) * ldg + offg + g);
        const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
        for (int a = 0; a < 8; a++) s[a] += __bfloat162float(e[a]);
      }
  uint4 o;
  bf16 *e = reinterpret_cast<bf16 *>(&o);
#pragma unroll
  for (int a = 0; a < 8; a++) e[a] = __float2bfloat16_rn(s[a]);
  *reinterpret_cast<uint4 *>(dC + (size_t)V * 32 + g) = o;
}

// dE[v, c] = (S[v, offs + c] + dP[parent, c] / children(parent)) * (E[v, offe + c] > 0)
// (the skip gradient, already masked, plus the pooled path's gradient)
__global__ void k_pool_back(dims f, dims c, const bf16 *dP, const bf16 *S, int lds, int offs, const bf16 *E, int lde,
                            int offe, bf16 *dE) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= f.V() * 4) return;
  int v = q >> 2, g = (q & 3) * 8;
  int z = v / (f.nx * f.ny), r = v - z * f.nx * f.ny, y = r / f.nx, x = r - y * f.nx;
  int X = x >> 1, Y = y >> 1, Z = z >> 1;
  int cnt = (min(f.nx, 2 * X + 2) - 2 * X) * (min(f.ny, 2 * Y + 2) - 2 * Y) * (min(f.nz, 2 * Z + 2) - 2 * Z);
  uint4 up = *reinterpret_cast<const uint4 *>(dP + (size_t)(X + c.nx * (Y + c.ny * Z)) * 32 + g);
  uint4 us = *reinterpret_cast<const uint4 *>(S + (size_t)v * lds + offs + g);
  uint4 ue = *reinterpret_cast<const uint4 *>(E + (size_t)v * lde + offe + g);
  const bf16 *ep = reinterpret_cast<const bf16 *>(&up), *es = reinterpret_cast<const bf16 *>(&us),
             *ee = reinterpret_cast<const bf16 *>(&ue);
  uint4 o;
  bf16 *eo = reinterpret_cast<bf16 *>(&o);
#pragma unroll
  for (int a = 0; a < 8; a++) {
    float val = __bfloat162float(es[a]) + __bfloat162float(ep[a]) / (float)cnt;
    eo[a] = __float2bfloat16_rn(__bfloat162float(ee[a]) > 0.f ? val : 0.f);
  }
  *reinterpret_cast<uint4 *>(dE + (size_t)v * 32 + g) = o;
}

// ---------------------------------------------------------- loss, Adam ----
// dY[v, c] = (Y[v, c] - T[v, c]) / V for c < 2, 0 for the other 14 channels;
// part[block] = sum of the block's squared errors
__global__ void k_loss(int V, const float *Y, const float *T, bf16 *dY, float *part) {
  __shared__ float sh[256];
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  float s = 0.f;
  if (v < V) {
    float e0 = Y[(size_t)v * COUT_HEAD] - T[2 * (size_t)v], e1 = Y[(size_t)v * COUT_HEAD + 1] - T[2 * (size_t)v + 1];
    s = e0 * e0 + e1 * e1;
    float inv = 1.0f / (float)V;
    uint4 z0 = make_uint4(0, 0, 0, 0);
    uint4 *d = reinterpret_cast<uint4 *>(dY + (size_t)v * 16);
    __nv_bfloat162 g = __floats2bfloat162_rn(e0 * inv, e1 * inv);
    uint4 first = z0;
    first.x = *reinterpret_cast<unsigned *>(&g);
    d[0] = first;
    d[1] = z0;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// out[0] (+)= scale * sum of the n partials (one warp, fixed order)
__global__ void k_sum_parts(int n, const float *part, double scale, double *out, int accumulate) {
  double t = 0.0;
  for (int k = threadIdx.x; k < n; k += 32) t += (double)part[k];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) out[0] = (accumulate ? out[0] : 0.0) + scale * t;
}

// Adam (Kingma and Ba, Algorithm 1) on the flat parameter array; the
// gradient is divided by `gdiv` (the number of samples accumulated)
__global__ void k_adam(int n, float *p, float *m, float *v, const float *g, float lr, float b1, float b2, float c1,
                       float c2, float eps, float gdiv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i] / gdiv;
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi; v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of one layer: Wf[t][o][c] = W[t][o][c]; Wb[26-t][c][o] = W[t][o][c]
// (Wb's o dimension padded to cob with zeros)
__global__ void k_pack(int co, int ci, int cb, const float *W, bf16 *Wf, bf16 *Wb) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 27 * co * ci) return;
  int t = q / (co * ci), r = q - t * co * ci, o = r / ci, c = r - o * ci;
  bf16 w = __float2bfloat16_rn(W[q]);
  Wf[q] = w;
  Wb[((size_t)(26 - t) * ci + c) * cb + o] = w;
}

// network input from FP32 features [V][8] -> BF16 [V][16]
__global__ void k_feat_in(int V, const float *F, bf16 *X) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  bf16 *o = X + (size_t)v * CIN_GPU;
  for (int c = 0; c < CIN_USED; c++) o[c] = __float2bfloat16_rn(F[(size_t)v * CIN_USED + c]);
  for (int c = CIN_USED; c < CIN_GPU; c++) o[c] = __float2bfloat16_rn(0.f);
}

// ------------------------------------------------------------ the net -----
struct level_bufs {
  dims d;
  dbuf<bf16> a, da, b, cat, p;          // encoder / decoder first-conv outputs, second decoder conv,
                                        // concat [up, skip] [V][64], pooled input
  dbuf<bf16> ga, gda, gb, gcat, ge, gp; // gradients
};

}  // namespace nn
using namespace nn;

struct sim_ws_s {
  cudaStream_t st = nullptr;
  size_t np = 0;                          // number of parameters (device layout)
  size_t woff[NLAYER], boff[NLAYER];      // offsets into the flat arrays
  size_t wfoff[NLAYER], wboff[NLAYER];    // offsets into the BF16 copies
  dbuf<float> P, M, Vm, G;                // master parameters, Adam moments, gradients
  dbuf<bf16> Wf, Wb;
  long long tstep = 0;                    // Adam steps taken
  int accum = 0;                          // samples accumulated in G
  // activations for the current grid
  dims cur = {0, 0, 0};
  level_bufs L[4];
  dbuf<bf16> X0, dY;
  dbuf<float> Y, part, lpart, T32, F32;
  dbuf<double> lsum;
  // dataset of (features, target) pairs taken from simulator solves
  struct sample { dims d; dbuf<bf16> X; dbuf<float> T; };
  std::vector<std::unique_ptr<sample>> data;
  size_t max_samples = 1u << 30;
  unsigned long long seed = 0;
  std::mutex use;                         // one caller at a time (activations are shared)
  bool tc = false;                        // tcgen05 convolutions (else mma.sync, the faster here)
  dbuf<int> err;                          // set by a kernel whose bounded wait gave up
  ~sim_ws_s() { if (st) cudaStreamDestroy(st); }
};

namespace nn {

static void ws_layout(sim_ws_s *w) {
  size_t o = 0, fo = 0, bo = 0;
  for (int l = 0; l < NLAYER; l++) {
    w->woff[l] = o; o += (size_t)27 * LAYERS[l].co * LAYERS[l].ci;
    w->boff[l] = o; o += LAYERS[l].co;
    w->wfoff[l] = fo; fo += (size_t)27 * LAYERS[l].co * LAYERS[l].ci;
    w->wboff[l] = bo; bo += (size_t)27 * LAYERS[l].ci * cob(l);
  }
  w->np = o;
  w->P.alloc(o); w->M.alloc(o); w->Vm.alloc(o); w->G.alloc(o);
  w->Wf.alloc(fo); w->Wb.alloc(bo);
}

static void ws_pack(sim_ws_s *w) {
  RS_CUDA(cudaMemsetAsync(w->Wb.p, 0, w->Wb.n * sizeof(bf16), w->st));
  for (int l = 0; l < NLAYER; l++) {
    int n = 27 * LAYERS[l].co * LAYERS[l].ci;
    k_pack<<<grid_for(n, 256), 256, 0, w->st>>>(LAYERS[l].co, LAYERS[l].ci, cob(l), w->P.p + w->woff[l],
                                                 w->Wf.p + w->wfoff[l], w->Wb.p + w->wboff[l]);
  }
  RS_LAUNCHED(NLAYER);
  RS_CHECK_LAUNCH();
}

template <int CI, int NT, int MODE>
static void conv_launch(sim_ws_s *w, dims d, const bf16 *X, int ldx, int offx, const bf16 *Wt, const float *bias,
                        int relu, void *out, int ldo, int offo, const bf16 *mask, int ldm, int offm) {
  static bool attr = false;
  int bytes = conv_smem<CI, NT>::BYTES;
  if (!attr) {
    RS_CUDA(cudaFuncSetAttribute(k_conv<CI, NT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    attr = true;
  }
  k_conv<CI, NT, MODE><<<grid_for(d.V(), CBM), 128, bytes, w->st>>>(d.nx, d.ny, d.nz, X, ldx, offx, Wt, bias, relu, out,
                                                                     ldo, offo, mask, ldm, offm);
  RS_LAUNCHED(1);
}

template <int CI, int NT, int MODE>
static void conv_halo_launch(sim_ws_s *w, dims d, const bf16 *X, int ldx, int offx, const bf16 *Wt, const float *bias,
                             int relu, void *out, int ldo, int offo) {
  static bool attr = false;
  int bytes = halo_smem<CI, NT>::BYTES;
  if (!attr) {
    RS_CUDA(cudaFuncSetAttribute(k_conv_halo<CI, NT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    attr = true;
  }
  unsigned tiles = (unsigned)(((d.nx + HX - 1) / HX) * ((d.ny + HY - 1) / HY) * ((d.nz + HZ - 1) / HZ));
  k_conv_halo<CI, NT, MODE><<<tiles, 128, bytes, w->st>>>(d.nx, d.ny, d.nz, X, ldx, offx, Wt, bias, relu, out, ldo,
                                                           offo);
  RS_LAUNCHED(1);
}

template <int CI, int CO, int MODE>
static void conv_tc_launch(sim_ws_s *w, dims d, const bf16 *X, int ldx, int offx, const bf16 *Wt, const float *bias,
                           int relu, void *out, int ldo, int offo, const bf16 *mask, int ldm, int offm) {
  static int per_sm = 0;                      // resident CTAs per SM for this instantiation
  static int sms = 0;
  int bytes = tc_smem<CI, CO>::BYTES;
  if (!per_sm) {
    RS_CUDA(cudaFuncSetAttribute(k_conv_tc<CI, CO, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    RS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    RS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_tc<CI, CO, MODE>, 128, bytes));
    if (per_sm < 1) per_sm = 1;
  }
  unsigned tiles = grid_for(d.V(), CBM), cap = (unsigned)(sms * per_sm), grid = tiles < cap ? tiles : cap;
  k_conv_tc<CI, CO, MODE><<<grid, 128, bytes, w->st>>>(d.nx, d.ny, d.nz, X, ldx, offx, Wt, bias, relu,
                                                                        reinterpret_cast<bf16 *>(out), ldo, offo, mask,
                                                                        ldm, offm, w->err.p);
  RS_LAUNCHED(1);
}

// forward conv of layer l: in (ld, off) -> out (ldo, offo)
static void fwd(sim_ws_s *w, int l, dims d, const bf16 *X, int ldx, int offx, void *out, int ldo, int offo) {
  const bf16 *Wt = w->Wf.p + w->wfoff[l];
  const float *b = w->P.p + w->boff[l];
  int ci = LAYERS[l].ci;
  if (l == HEAD) conv_halo_launch<32, 1, 1>(w, d, X, ldx, offx, Wt, b, 0, out, ldo, offo);
  else if (w->tc) {
    if (ci == 16) conv_tc_launch<16, 32, 0>(w, d, X, ldx, offx, Wt, b, 1, out, ldo, offo, nullptr, 0, 0);
    else if (ci == 32) conv_tc_launch<32, 32, 0>(w, d, X, ldx, offx, Wt, b, 1, out, ldo, offo, nullptr, 0, 0);
    else conv_tc_launch<64, 32, 0>(w, d, X, ldx, offx, Wt, b, 1, out, ldo, offo, nullptr, 0, 0);
  }
  else if (ci == 16) conv_halo_launch<16, 4, 0>(w, d, X, ldx, offx, Wt, b, 1, out, ldo, offo);
  else if (ci == 32) conv_halo_launch<32, 4, 0>(w, d, X, ldx, offx, Wt, b, 1, out, ldo, offo);
  else conv_halo_launch<64, 4, 0>(w, d, X, ldx, offx, Wt, b, 1, out, ldo, offo);
}

// data gradient of layer l: dZ (ldz, offz) -> dX (ldo, offo), masked by the
// layer's input (mask != nullptr) when that input came out of a ReLU
static void bwd_data(sim_ws_s *w, int l, dims d, const bf16 *dZ, int ldz, int offz, bf16 *out, int ldo, int offo,
                     const bf16 *mask, int ldm, int offm) {
  const bf16 *Wt = w->Wb.p + w->wboff[l];
  int ci = LAYERS[l].ci;
  if (w->tc && l != C00) {
    if (l == HEAD) {
      if (mask) conv_tc_launch<16, 32, 2>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
      else conv_tc_launch<16, 32, 3>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
    } else if (ci == 64) {
      if (mask) conv_tc_launch<32, 64, 2>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
      else conv_tc_launch<32, 64, 3>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
    } else {
      if (mask) conv_tc_launch<32, 32, 2>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
      else conv_tc_launch<32, 32, 3>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
    }
    return;
  }
  if (l == HEAD) {     // input: dY with 16 channels; output 32
    if (mask) conv_launch<16, 4, 2>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
    else conv_launch<16, 4, 3>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
  } else if (ci == 64) {
    if (mask) conv_launch<32, 8, 2>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
    else conv_launch<32, 8, 3>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
  } else if (ci == 32) {
    if (mask) conv_launch<32, 4, 2>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
    else conv_launch<32, 4, 3>(w, d, dZ, ldz, offz, Wt, nullptr, 0, out, ldo, offo, mask, ldm, offm);
  } else {
    RS_FAIL(SIM_ERR_ARG, "no data gradient for the input layer");
  }
}

template <int CI, int MT>
static void wgrad_launch(sim_ws_s *w, int l, dims d, const bf16 *X, int ldx, int offx, const bf16 *dZ, int ldz, int offz) {
  static bool attr = false;
  int bytes = wg_smem<CI, MT>::BYTES;
  if (!attr) {
    RS_CUDA(cudaFuncSetAttribute(k_conv_wgrad<CI, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    attr = true;
  }
  int co = LAYERS[l].co;
  int nchunk = (d.V() + WCH * WIT - 1) / (WCH * WIT);
  size_t need = (size_t)27 * nchunk * co * CI;
  w->part.ensure(need + (size_t)nchunk * co);
  float *bpart = w->part.p + need;
  k_conv_wgrad<CI, MT><<<dim3(nchunk, 27), 256, bytes, w->st>>>(d.nx, d.ny, d.nz, X, ldx, offx, dZ, ldz, offz, co,
                                                                 w->part.p, bpart);
  int per_tap = co * CI;
  k_wgrad_reduce<<<grid_for(27 * per_tap + co, 256), 256, 0, w->st>>>(nchunk, per_tap, w->part.p, bpart, co,
                                                                       w->G.p + w->woff[l], w->G.p + w->boff[l]);
  RS_LAUNCHED(2);
}

static void wgrad(sim_ws_s *w, int l, dims d, const bf16 *X, int ldx, int offx, const bf16 *dZ, int ldz, int offz) {
  int ci = LAYERS[l].ci;
  if (l == HEAD) wgrad_launch<32, 1>(w, l, d, X, ldx, offx, dZ, ldz, offz);
  else if (ci == 16) wgrad_launch<16, 2>(w, l, d, X, ldx, offx, dZ, ldz, offz);
  else if (ci == 32) wgrad_launch<32, 2>(w, l, d, X, ldx, offx, dZ, ldz, offz);
  else wgrad_launch<64, 2>(w, l, d, X, ldx, offx, dZ, ldz, offz);
}

static void ensure_dims(sim_ws_s *w, dims d) {
  if (d.nx == w->cur.nx && d.ny == w->cur.ny && d.nz == w->cur.nz) return;
  dims c = d;
  for (int k = 0; k < 4; k++) {
    level_bufs &B = w->L[k];
    B.d = c;
    size_t V = c.V();
    B.a.alloc(V * 32); B.da.alloc(V * 32); B.b.alloc(V * 32); B.cat.alloc(V * 64); B.p.alloc(V * 32);
    B.ga.alloc(V * 32); B.gda.alloc(V * 32); B.gb.alloc(V * 32); B.gcat.alloc(V * 64); B.ge.alloc(V * 32);
    B.gp.alloc(V * 32);
    c = coarse(c);
  }
  size_t V = d.V();
  w->X0.alloc(V * CIN_GPU); w->dY.alloc(V * 16); w->Y.alloc(V * COUT_HEAD);
  w->lpart.alloc(grid_for(V, 256));
  w->cur = d;
}

// Forward pass on w->X0 (BF16 [V][16]) -> w->Y (FP32 [V][8]).
// Level k buffers: a = first encoder conv, cat = [up, skip] (skip = second
// encoder conv), p = pooled input (levels 1..3), da = first decoder conv,
// b = second decoder conv (the bottom's second conv at level 3).
static void forward(sim_ws_s *w) {
  level_bufs *L = w->L;
  fwd(w, C00, L[0].d, w->X0.p, CIN_GPU, 0, L[0].a.p, 32, 0);
  fwd(w, C01, L[0].d, L[0].a.p, 32, 0, L[0].cat.p, 64, 32);
  for (int k = 1; k <= 3; k++) {
    k_pool<<<grid_for((size_t)L[k].d.V() * 4, 256), 256, 0, w->st>>>(L[k - 1].d, L[k].d, L[k - 1].cat.p, 64, 32, L[k].p.p);
    RS_LAUNCHED(1);
    int c0 = k == 1 ? C10 : k == 2 ? C20 : C30;
    fwd(w, c0, L[k].d, L[k].p.p, 32, 0, L[k].a.p, 32, 0);
    if (k < 3) fwd(w, c0 + 1, L[k].d, L[k].a.p, 32, 0, L[k].cat.p, 64, 32);
    else fwd(w, c0 + 1, L[k].d, L[k].a.p, 32, 0, L[k].b.p, 32, 0);
  }
  for (int k = 2; k >= 0; k--) {
    k_up<<<grid_for((size_t)L[k].d.V() * 4, 256), 256, 0, w->st>>>(L[k].d, L[k + 1].d, L[k + 1].b.p, L[k].cat.p, 64, 0);
    RS_LAUNCHED(1);
    int d0 = k == 2 ? D20 : k == 1 ? D10 : D00;
    fwd(w, d0, L[k].d, L[k].cat.p, 64, 0, L[k].da.p, 32, 0);
    fwd(w, d0 + 1, L[k].d, L[k].da.p, 32, 0, L[k].b.p, 32, 0);
  }
  fwd(w, HEAD, L[0].d, L[0].b.p, 32, 0, w->Y.p, COUT_HEAD, 0);
  RS_CHECK_LAUNCH();
}

// loss against T32 ([V][2]) accumulated into lsum (scaled 0.5/V); gradients
// accumulated into G.  Uses the activations of the last forward().
static void backward(sim_ws_s *w, const float *T) {
  level_bufs *L = w->L;
  int V = L[0].d.V();
  k_loss<<<grid_for(V, 256), 256, 0, w->st>>>(V, w->Y.p, T, w->dY.p, w->lpart.p);
  k_sum_parts<<<1, 32, 0, w->st>>>((int)grid_for(V, 256), w->lpart.p, 0.5 / V, w->lsum.p, 1);
  RS_LAUNCHED(2);
  // head: input b0, output dY
  wgrad(w, HEAD, L[0].d, L[0].b.p, 32, 0, w->dY.p, 16, 0);
  bwd_data(w, HEAD, L[0].d, w->dY.p, 16, 0, L[0].gb.p, 32, 0, L[0].b.p, 32, 0);
  // decoder, finest level first
  for (int k = 0; k <= 2; k++) {
    int d0 = k == 2 ? D20 : k == 1 ? D10 : D00;
    // second decoder conv: input da, output gradient gb
    wgrad(w, d0 + 1, L[k].d, L[k].da.p, 32, 0, L[k].gb.p, 32, 0);
    bwd_data(w, d0 + 1, L[k].d, L[k].gb.p, 32, 0, L[k].gda.p, 32, 0, L[k].da.p, 32, 0);
    // first decoder conv: input cat, output gradient gda
    wgrad(w, d0, L[k].d, L[k].cat.p, 64, 0, L[k].gda.p, 32, 0);
    bwd_data(w, d0, L[k].d, L[k].gda.p, 32, 0, L[k].gcat.p, 64, 0, L[k].cat.p, 64, 0);
    // up-sampled half -> gradient of the coarser level's output (gb there)
    k_up_back<<<grid_for((size_t)L[k + 1].d.V() * 4, 256), 256, 0, w->st>>>(L[k].d, L[k + 1].d, L[k].gcat.p, 64, 0,
                                                                           L[k + 1].gb.p);
    RS_LAUNCHED(1);
  }
  // bottom: c31 (input a3, output b3), c30 (input p3)
  wgrad(w, C31, L[3].d, L[3].a.p, 32, 0, L[3].gb.p, 32, 0);
  bwd_data(w, C31, L[3].d, L[3].gb.p, 32, 0, L[3].ga.p, 32, 0, L[3].a.p, 32, 0);
  wgrad(w, C30, L[3].d, L[3].p.p, 32, 0, L[3].ga.p, 32, 0);
  bwd_data(w, C30, L[3].d, L[3].ga.p, 32, 0, L[3].gp.p, 32, 0, nullptr, 0, 0);
  // encoder, coarse to fine: ge(k) = mask * (skip part of gcat(k) + pool-back of gp(k+1))
  for (int k = 2; k >= 0; k--) {
    k_pool_back<<<grid_for((size_t)L[k].d.V() * 4, 256), 256, 0, w->st>>>(L[k].d, L[k + 1].d, L[k + 1].gp.p,
                                                                         L[k].gcat.p, 64, 32, L[k].cat.p, 64, 32,
                                                                         L[k].ge.p);
    RS_LAUNCHED(1);
    int c0 = k == 2 ? C20 : k == 1 ? C10 : C00;
    wgrad(w, c0 + 1, L[k].d, L[k].a.p, 32, 0, L[k].ge.p, 32, 0);
    bwd_data(w, c0 + 1, L[k].d, L[k].ge.p, 32, 0, L[k].ga.p, 32, 0, L[k].a.p, 32, 0);
    if (k > 0) {
      wgrad(w, c0, L[k].d, L[k].p.p, 32, 0, L[k].ga.p, 32, 0);
      bwd_data(w, c0, L[k].d, L[k].ga.p, 32, 0, L[k].gp.p, 32, 0, nullptr, 0, 0);
    } else {
      wgrad(w, C00, L[0].d, w->X0.p, CIN_GPU, 0, L[0].ga.p, 32, 0);
    }
  }
  RS_CHECK_LAUNCH();
  w->accum++;
}

static void zero_grad(sim_ws_s *w) {
  RS_CUDA(cudaMemsetAsync(w->G.p, 0, w->np * sizeof(float), w->st));
  w->accum = 0;
}

static void adam(sim_ws_s *w, double lr) {
  if (w->accum == 0) return;
  w->tstep++;
  const double b1 = 0.9, b2 = 0.999;
  float c1 = (float)(1.0 - std::pow(b1, (double)w->tstep)), c2 = (float)(1.0 - std::pow(b2, (double)w->tstep));
  k_adam<<<grid_for(w->np, 256), 256, 0, w->st>>>((int)w->np, w->P.p, w->M.p, w->Vm.p, w->G.p, (float)lr, (float)b1,
                                                 (float)b2, c1, c2, 1e-8f, (float)w->accum);
  RS_LAUNCHED(1);
  ws_pack(w);
  zero_grad(w);
}

// splitmix64 (Steele, Lea and Flood 2014) and a Box-Muller normal draw for
// the He initialisation
static inline uint64_t smix(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline double unif(uint64_t &s) { return ((smix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

}  // namespace nn

// ---------------------------------------------------------------- ABI -----
#define ABI_BEGIN try {
#define ABI_END                                                       \
  }                                                                   \
  catch (const rs_error &e) { return e.code; }                        \
  catch (const std::bad_alloc &) { rs_set_error("host allocation failed"); return SIM_ERR_OOM; } \
  catch (...) { rs_set_error("unexpected exception"); return SIM_ERR_CUDA; }                       \
  return SIM_OK;

// parameter count in the exported layout: per layer W[27][Co][Ci] (Ci = 8 for
// the input layer) then b[Co]
static size_t export_count() {
  size_t n = 0;
  for (int l = 0; l < NLAYER; l++) n += (size_t)27 * LAYERS[l].co * ci_true(l) + LAYERS[l].co;
  return n;
}

// a tensor-core kernel whose bounded wait gave up leaves a flag; report it
static void check_err(sim_ws_s *w) {
  int e = 0;
  RS_CUDA(cudaMemcpyAsync(&e, w->err.p, sizeof(int), cudaMemcpyDeviceToHost, w->st));
  RS_CUDA(cudaStreamSynchronize(w->st));
  if (e) {
    RS_CUDA(cudaMemsetAsync(w->err.p, 0, sizeof(int), w->st));
    RS_FAIL(SIM_ERR_TIMEOUT, "warm-start network: a tensor-core pipeline wait gave up");
  }
}

extern "C" sim_status sim_ws_create(sim_ws_t *out, unsigned long long seed) {
  ABI_BEGIN
  if (!out) RS_FAIL(SIM_ERR_ARG, "sim_ws_create: NULL argument");
  *out = nullptr;
  std::unique_ptr<sim_ws_s> w(new sim_ws_s());
  RS_CUDA(cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking));
  ws_layout(w.get());
  w->seed = seed;
  // He-normal weights (std sqrt(2 / (27 ci))), zero biases; padding channels
  // zero; the head starts at zero, so an untrained network predicts no
  // correction
  std::vector<float> h(w->np, 0.f);
  uint64_t s = seed;
  for (int l = 0; l < HEAD; l++) {
    int co = LAYERS[l].co, ci = LAYERS[l].ci, ct = ci_true(l);
    double sd = std::sqrt(2.0 / (27.0 * ct));
    for (int t = 0; t < 27; t++)
      for (int o = 0; o < co; o++)
        for (int c = 0; c < ct; c++) {
          double u1 = unif(s), u2 = unif(s);
          h[w->woff[l] + ((size_t)t * co + o) * ci + c] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
  }
  RS_CUDA(cudaMemcpyAsync(w->P.p, h.data(), w->np * sizeof(float), cudaMemcpyHostToDevice, w->st));
  RS_CUDA(cudaMemsetAsync(w->M.p, 0, w->np * sizeof(float), w->st));
  RS_CUDA(cudaMemsetAsync(w->Vm.p, 0, w->np * sizeof(float), w->st));
  w->lsum.alloc(2);
  w->err.alloc(1);
  RS_CUDA(cudaMemsetAsync(w->err.p, 0, sizeof(int), w->st));
  zero_grad(w.get());
  ws_pack(w.get());
  RS_CUDA(cudaStreamSynchronize(w->st));
  *out = w.release();
  ABI_END
}

extern "C" void sim_ws_destroy(sim_ws_t w) { delete w; }

extern "C" sim_status sim_ws_use_tcgen05(sim_ws_t w, int on) {
  ABI_BEGIN
  if (!w) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  std::lock_guard<std::mutex> guard(w->use);
  w->tc = on != 0;
  ABI_END
}

// which = 0: master parameters, 1: accumulated gradients (divided by the
// number of samples accumulated, i.e. the mean over the batch)
extern "C" sim_status sim_ws_params(sim_ws_t w, int which, float *dst, size_t n, size_t *needed) {
  ABI_BEGIN
  if (!w || (which != 0 && which != 1)) RS_FAIL(SIM_ERR_ARG, "sim_ws_params: bad argument");
  size_t ne = export_count();
  if (needed) *needed = ne;
  if (!dst) return SIM_OK;
  if (n < ne) RS_FAIL(SIM_ERR_ARG, "sim_ws_params: buffer holds %zu of %zu values", n, ne);
  std::vector<float> h = d2h(which == 0 ? w->P.p : w->G.p, w->np, w->st);
  float div = which == 1 && w->accum > 0 ? (float)w->accum : 1.f;
  size_t q = 0;
  for (int l = 0; l < NLAYER; l++) {
    int co = LAYERS[l].co, ci = LAYERS[l].ci, ct = ci_true(l);
    for (int t = 0; t < 27; t++)
      for (int o = 0; o < co; o++)
        for (int c = 0; c < ct; c++) dst[q++] = h[w->woff[l] + ((size_t)t * co + o) * ci + c] / div;
    for (int o = 0; o < co; o++) dst[q++] = h[w->boff[l] + o] / div;
  }
  ABI_END
}

extern "C" sim_status sim_ws_set_params(sim_ws_t w, const float *src, size_t n) {
  ABI_BEGIN
  if (!w || !src) RS_FAIL(SIM_ERR_ARG, "sim_ws_set_params: NULL argument");
  size_t ne = export_count();
  if (n != ne) RS_FAIL(SIM_ERR_ARG, "sim_ws_set_params: expected %zu values, got %zu", ne, n);
  std::vector<float> h(w->np, 0.f);
  size_t q = 0;
  for (int l = 0; l < NLAYER; l++) {
    int co = LAYERS[l].co, ci = LAYERS[l].ci, ct = ci_true(l);
    for (int t = 0; t < 27; t++)
      for (int o = 0; o < co; o++)
        for (int c = 0; c < ct; c++) h[w->woff[l] + ((size_t)t * co + o) * ci + c] = src[q++];
    for (int o = 0; o < co; o++) h[w->boff[l] + o] = src[q++];
  }
  RS_CUDA(cudaMemcpyAsync(w->P.p, h.data(), w->np * sizeof(float), cudaMemcpyHostToDevice, w->st));
  RS_CUDA(cudaMemsetAsync(w->M.p, 0, w->np * sizeof(float), w->st));
  RS_CUDA(cudaMemsetAsync(w->Vm.p, 0, w->np * sizeof(float), w->st));
  w->tstep = 0;
  zero_grad(w);
  ws_pack(w);
  RS_CUDA(cudaStreamSynchronize(w->st));
  ABI_END
}

static void load_features(sim_ws_s *w, dims d, const float *feat) {
  ensure_dims(w, d);
  size_t V = d.V();
  w->F32.ensure(V * CIN_USED);
  RS_CUDA(cudaMemcpyAsync(w->F32.p, feat, V * CIN_USED * sizeof(float), cudaMemcpyDefault, w->st));
  k_feat_in<<<grid_for(V, 256), 256, 0, w->st>>>((int)V, w->F32.p, w->X0.p);
  RS_LAUNCHED(1);
}

extern "C" sim_status sim_ws_forward(sim_ws_t w, int nx, int ny, int nz, const float *feat, float *y) {
  ABI_BEGIN
  if (!w || !feat || !y || nx < 1 || ny < 1 || nz < 1) RS_FAIL(SIM_ERR_ARG, "sim_ws_forward: bad argument");
  dims d = {nx, ny, nz};
  load_features(w, d, feat);
  forward(w);
  RS_CUDA(cudaMemcpyAsync(y, w->Y.p, (size_t)d.V() * COUT_HEAD * sizeof(float), cudaMemcpyDefault, w->st));
  RS_CUDA(cudaStreamSynchronize(w->st));
  check_err(w);
  ABI_END
}

// Forward, loss and backward for one sample; gradients are added to the
// accumulated ones (sim_ws_zero_grad clears them) and *loss receives this
// sample's loss.
extern "C" sim_status sim_ws_backward(sim_ws_t w, int nx, int ny, int nz, const float *feat, const float *target,
                                      double *loss) {
  ABI_BEGIN
  if (!w || !feat || !target || nx < 1 || ny < 1 || nz < 1) RS_FAIL(SIM_ERR_ARG, "sim_ws_backward: bad argument");
  dims d = {nx, ny, nz};
  load_features(w, d, feat);
  size_t V = d.V();
  w->T32.ensure(V * NPRED);
  RS_CUDA(cudaMemcpyAsync(w->T32.p, target, V * NPRED * sizeof(float), cudaMemcpyDefault, w->st));
  forward(w);
  RS_CUDA(cudaMemsetAsync(w->lsum.p, 0, sizeof(double), w->st));
  backward(w, w->T32.p);
  double l = 0.0;
  RS_CUDA(cudaMemcpyAsync(&l, w->lsum.p, sizeof(double), cudaMemcpyDeviceToHost, w->st));
  RS_CUDA(cudaStreamSynchronize(w->st));
  check_err(w);
  if (loss) *loss = l;
  ABI_END
}

extern "C" sim_status sim_ws_zero_grad(sim_ws_t w) {
  ABI_BEGIN
  if (!w) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  zero_grad(w);
  RS_CUDA(cudaStreamSynchronize(w->st));
  ABI_END
}

extern "C" sim_status sim_ws_adam(sim_ws_t w, double lr) {
  ABI_BEGIN
  if (!w || !(lr > 0)) RS_FAIL(SIM_ERR_ARG, "sim_ws_adam: bad argument");
  adam(w, lr);
  RS_CUDA(cudaStreamSynchronize(w->st));
  ABI_END
}

extern "C" sim_status sim_ws_dataset(sim_ws_t w, int *n_samples) {
  ABI_BEGIN
  if (!w || !n_samples) RS_FAIL(SIM_ERR_ARG, "NULL argument");
  *n_samples = (int)w->data.size();
  ABI_END
}

// Epochs over the recorded samples in a seeded random order, Adam step every
// `batch` samples; *mean_loss = mean sample loss of the last epoch.
extern "C" sim_status sim_ws_train(sim_ws_t w, int epochs, int batch, double lr, unsigned long long seed,
                                   double *mean_loss) {
  ABI_BEGIN
  if (!w || epochs < 0 || batch < 1 || !(lr > 0)) RS_FAIL(SIM_ERR_ARG, "sim_ws_train: bad argument");
  int n = (int)w->data.size();
  if (n == 0) RS_FAIL(SIM_ERR_STATE, "sim_ws_train: no recorded samples");
  std::vector<int> order(n);
  uint64_t s = seed;
  double last = 0.0;
  zero_grad(w);
  for (int e = 0; e < epochs; e++) {
    for (int k = 0; k < n; k++) order[k] = k;
    for (int k = n - 1; k > 0; k--) std::swap(order[k], order[(int)(smix(s) % (uint64_t)(k + 1))]);   // Fisher-Yates
    RS_CUDA(cudaMemsetAsync(w->lsum.p, 0, sizeof(double), w->st));
    for (int k = 0; k < n; k++) {
      auto &S = *w->data[order[k]];
      ensure_dims(w, S.d);
      RS_CUDA(cudaMemcpyAsync(w->X0.p, S.X.p, (size_t)S.d.V() * CIN_GPU * sizeof(bf16), cudaMemcpyDeviceToDevice, w->st));
      forward(w);
      backward(w, S.T.p);
      if (w->accum == batch || k == n - 1) adam(w, lr);
    }
    double l = 0.0;
    RS_CUDA(cudaMemcpyAsync(&l, w->lsum.p, sizeof(double), cudaMemcpyDeviceToHost, w->st));
    RS_CUDA(cudaStreamSynchronize(w->st));
    check_err(w);
    last = l / n;
  }
  if (mean_loss) *mean_loss = last;
  ABI_END
}

// mean loss over the recorded samples with the current weights (no update)
extern "C" sim_status sim_ws_eval(sim_ws_t w, double *mean_loss) {
  ABI_BEGIN
  if (!w || !mean_loss) RS_FAIL(SIM_ERR_ARG, "NULL argument");
  int n = (int)w->data.size();
  if (n == 0) RS_FAIL(SIM_ERR_STATE, "sim_ws_eval: no recorded samples");
  RS_CUDA(cudaMemsetAsync(w->lsum.p, 0, sizeof(double), w->st));
  for (int k = 0; k < n; k++) {
    auto &S = *w->data[k];
    ensure_dims(w, S.d);
    RS_CUDA(cudaMemcpyAsync(w->X0.p, S.X.p, (size_t)S.d.V() * CIN_GPU * sizeof(bf16), cudaMemcpyDeviceToDevice, w->st));
    forward(w);
    int V = S.d.V();
    k_loss<<<grid_for(V, 256), 256, 0, w->st>>>(V, w->Y.p, S.T.p, w->dY.p, w->lpart.p);
    k_sum_parts<<<1, 32, 0, w->st>>>((int)grid_for(V, 256), w->lpart.p, 0.5 / V, w->lsum.p, 1);
    RS_LAUNCHED(2);
  }
  double l = 0.0;
  RS_CUDA(cudaMemcpyAsync(&l, w->lsum.p, sizeof(double), cudaMemcpyDeviceToHost, w->st));
  RS_CUDA(cudaStreamSynchronize(w->st));
  check_err(w);
  *mean_loss = l / n;
  ABI_END
}

// ------------------------------------------------ simulator integration ---
// Features of the current system, on the simulator's stream: X [n][16] BF16,
// from the decoupled right-hand side b (the Newton residual), ln k, s_w and
// the previous solve's update yp (cell rows; each vector component over its
// rms over the cells; channels 6-7 are zero):
//   sc[0], sc[1] = rms of b (pressure / saturation rows),
//   sc[2], sc[3] = rms of the solved update (recording only: the target's scales),
//   sc[4], sc[5] = rms of yp (0 when there is no previous update).
__global__ void k_ws_features(int n, const double *b, const double *kx, const double *sw, const double *yp,
                              const double *sc, bf16 *X) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  auto q = [](double a, double s) { return s > 0.0 ? (float)(a / s) : 0.f; };
  float f[8];
  f[0] = q(b[2 * (size_t)c], sc[0]);
  f[1] = q(b[2 * (size_t)c + 1], sc[1]);
  f[2] = (float)((log(kx[c]) - 4.0) * 0.5);
  f[3] = (float)((sw[c] - 0.5) * 4.0);
  f[4] = q(yp[2 * (size_t)c], sc[4]);
  f[5] = q(yp[2 * (size_t)c + 1], sc[5]);
  f[6] = 0.f;
  f[7] = 0.f;
  bf16 *o = X + (size_t)c * CIN_GPU;
#pragma unroll
  for (int a = 0; a < 8; a++) o[a] = __float2bfloat16_rn(f[a]);
#pragma unroll
  for (int a = 8; a < CIN_GPU; a++) o[a] = __float2bfloat16_rn(0.f);
}

// The network predicts the update's shape, each component with unit rms:
// two candidate vectors, its pressure part dp = (Y[c][0], 0) and its
// saturation part ds = (0, Y[c][1]) for cells, 0 for well rows (the least-
// squares fit of the initial guess sets both scales)
__global__ void k_ws_predict(int n, int nb, const float *Y, double *dp, double *ds) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * nb) return;
  int c = i >> 1, a = i & 1;
  double v = c < n ? (double)Y[(size_t)c * COUT_HEAD + a] : 0.0;
  dp[i] = a == 0 ? v : 0.0;
  ds[i] = a == 1 ? v : 0.0;
}

// T[c][a] = y[2c + a] / rms(y_a) (the training target of this system)
__global__ void k_ws_target(int n, const double *y, const double *sc, float *T) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  double s = sc[2 + (i & 1)];
  T[i] = s > 0.0 ? (float)(y[i] / s) : 0.f;
}

// rms over the n cells of the two interleaved components of v -> out[0], out[1]
__global__ void k_rms2(int n, const double *v, double *out) {
  __shared__ double sh[2][1024];
  double s0 = 0.0, s1 = 0.0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double a = v[2 * (size_t)c], b = v[2 * (size_t)c + 1];
    s0 += a * a; s1 += b * b;
  }
  sh[0][threadIdx.x] = s0; sh[1][threadIdx.x] = s1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { sh[0][threadIdx.x] += sh[0][threadIdx.x + o]; sh[1][threadIdx.x] += sh[1][threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = sqrt(sh[0][0] / n); out[1] = sqrt(sh[1][0] / n); }
}

void ws_rms2(int n, const double *v, double *out, cudaStream_t s) {
  k_rms2<<<1, 1024, 0, s>>>(n, v, out);
  RS_LAUNCHED(1);
}

// predicted update as two candidates in y (2 x 2 nb, FP64, device: pressure
// part, then saturation part) for the system whose decoupled right-hand side
// is b; yp, sc as above (device)
void ws_predict(sim_ws_s *w, int nx, int ny, int nz, int nb, const double *b, const double *kx, const double *sw,
                const double *yp, const double *sc, double *y, cudaStream_t s) {
  std::lock_guard<std::mutex> guard(w->use);
  dims d = {nx, ny, nz};
  ensure_dims(w, d);
  int n = d.V();
  // the network runs on its own stream, ordered after the simulator's work
  cudaEvent_t ev;
  RS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  k_ws_features<<<grid_for(n, 256), 256, 0, s>>>(n, b, kx, sw, yp, sc, w->X0.p);
  RS_LAUNCHED(1);
  RS_CUDA(cudaEventRecord(ev, s));
  RS_CUDA(cudaStreamWaitEvent(w->st, ev, 0));
  forward(w);
  RS_CUDA(cudaEventRecord(ev, w->st));
  RS_CUDA(cudaStreamWaitEvent(s, ev, 0));
  RS_CUDA(cudaEventDestroy(ev));
  k_ws_predict<<<grid_for(2 * nb, 256), 256, 0, s>>>(n, nb, w->Y.p, y, y + 2 * (size_t)nb);
  RS_LAUNCHED(1);
}

// append (features, target) of a solved system to the dataset
void ws_record(sim_ws_s *w, int nx, int ny, int nz, const double *b, const double *kx, const double *sw,
               const double *yp, const double *sc, const double *y, cudaStream_t s) {
  std::lock_guard<std::mutex> guard(w->use);
  if (w->data.size() >= w->max_samples) return;
  dims d = {nx, ny, nz};
  int n = d.V();
  std::unique_ptr<sim_ws_s::sample> S(new sim_ws_s::sample());
  S->d = d;
  S->X.alloc((size_t)n * CIN_GPU);
  S->T.alloc((size_t)n * NPRED);
  k_ws_features<<<grid_for(n, 256), 256, 0, s>>>(n, b, kx, sw, yp, sc, S->X.p);
  k_ws_target<<<grid_for(2 * n, 256), 256, 0, s>>>(n, y, sc, S->T.p);
  RS_LAUNCHED(2);
  RS_CUDA(cudaStreamSynchronize(s));       // the sample is complete before another stream reads it
  w->data.push_back(std::move(S));
}

cudaStream_t ws_stream(sim_ws_s *w) { return w->st; }
