// Kernels of the learned right preconditioner: a 3-level 3D U-Net (16/32/64 channels, 3x3x3
// convolutions, 2x average pooling, 2x2x2 transposed convolutions, skip concatenation, 1x1x1
// head), BF16 activations and weights with FP32 accumulation, NDHWC layout (channels innermost,
// voxel index x + nx*(y + ny*z)).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

typedef __nv_bfloat16 bf16;

namespace unet {

// ------------------------------------------------------------------------------------------------
// 3x3x3 convolution, stride 1, zero padding 1, as an implicit GEMM on the tensor cores:
//   out[v][co] = act( bias[co] + sum_{tap, ci} in[v + off(tap)][ci] * W[tap][co][ci] )
// M = output voxels (a CTA owns 32 x TY of them per plane and marches along z, a warp 16 or 32
// along x), N = output channels (NC per CTA), K = 27 * CIN.  Input halo planes and the CTA's weight
// slice are staged in shared memory and fed to mma.sync m16n8k16 (bf16 x bf16 -> f32) through
// ldmatrix.
// Two input sources implement the skip concatenation (channels [0, c1) from in1, [c1, CIN) from
// in2); two outputs split the output channels ([0, o1) to out1, the rest to out2).  The backward
// data pass (dgrad) is this same kernel on flipped, transposed weights.
// ------------------------------------------------------------------------------------------------
struct ConvArgs {
  const bf16* in1;
  const bf16* in2;
  int c1, c2;        // channels of the two inputs (c1 + c2 = CIN)
  const bf16* w;     // [27][cout][CIN]
  const float* bias; // [cout] or null
  bf16* out1;
  bf16* out2;
  int o1, o2;        // channels of the two outputs (o1 + o2 = cout)
  int cout;
  int nx, ny, nz;
  int relu;
};

constexpr int CX = 32;  // output voxels per CTA along x

__device__ inline uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ inline void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ inline void cp_async16(uint32_t dst, const void* src, int src_bytes) {  // src_bytes 0: zero fill
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The CTA owns a 32 x TY tile of output voxels in (x, y) and a chunk of tz planes along z, for NC
// output channels.  Its weight slice is staged once; input halo planes (34 x (TY+2) voxels x CIN
// channels, rows padded by 8 channels so ldmatrix is conflict-free) live in a ring of 4: planes
// z-1, z, z+1 are read while plane z+2 is copied in with cp.async (zero fill outside the grid).
// Each of the 8 warps owns TY/4 m16 tiles (16 voxels along x) and all NC channels; the B fragments
// of a (tap, k-chunk) are loaded once and used for all of the warp's tiles.
template <int CIN, int NC, int TY>
struct Conv3Shape {
  static constexpr int RS = CIN + 8;          // padded channel stride (bf16) of a staged voxel
  static constexpr int PX = CX + 2, PY = TY + 2;
  static constexpr int PLANE = PX * PY * RS;  // bf16 per staged halo plane
  static constexpr int MT = TY / 4;           // m16 tiles per warp (2 * TY tiles over 8 warps)
  static constexpr int smem() { return (27 * NC * RS + 4 * PLANE) * (int)sizeof(bf16); }
};

template <int CIN, int NC, int TY>
__global__ void __launch_bounds__(256) conv3_kernel(ConvArgs a, int tz) {
  using SH = Conv3Shape<CIN, NC, TY>;
  constexpr int RS = SH::RS, PX = SH::PX, PY = SH::PY, MT = SH::MT, CH8 = CIN / 8;
  static_assert(TY % 4 == 0 && CIN % 16 == 0 && NC % 16 == 0, "conv3 tile shape");
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* w_s = (bf16*)smem;             // [27][NC][RS]
  bf16* ring = w_s + 27 * NC * RS;     // [4][PY][PX][RS]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * CX, y0 = blockIdx.y * TY;
  const int nblk_n = (a.cout + NC - 1) / NC;
  const int zc = blockIdx.z / nblk_n, n0 = (blockIdx.z % nblk_n) * NC;
  const int z0 = zc * tz, z1 = min(a.nz, z0 + tz);
  if (z0 >= z1) return;

  // plane p goes to ring slot (p - (z0 - 1)) % 4
  auto load_plane = [&](int p) {
    bf16* dst = ring + ((p - (z0 - 1)) & 3) * SH::PLANE;
    for (int q = tid; q < PX * PY * CH8; q += 256) {
      const int c8 = q % CH8, vox = q / CH8;
      const int hx = vox % PX, hy = vox / PX;
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
      const bool in = gx >= 0 && gy >= 0 && p >= 0 && gx < a.nx && gy < a.ny && p < a.nz;
      const void* src = a.in1;  // a valid address even when nothing is read
      if (in) {
        const long long gv = gx + (long long)a.nx * (gy + (long long)a.ny * p);
        const int c = c8 * 8;
        src = c < a.c1 ? (const void*)(a.in1 + gv * a.c1 + c) : (const void*)(a.in2 + gv * a.c2 + (c - a.c1));
      }
      cp_async16(smem_addr(dst + vox * RS + c8 * 8), src, in ? 16 : 0);
    }
  };
  // weights (output channels n0 .. n0+NC-1) and the first three planes: one copy group
  for (int q = tid; q < 27 * NC * CH8; q += 256) {
    const int c8 = q % CH8, row = q / CH8;
    const int tap = row / NC, n = row % NC;
    const bool in = n0 + n < a.cout;
    const void* src = in ? (const void*)(a.w + ((long long)tap * a.cout + n0 + n) * CIN + c8 * 8) : (const void*)a.w;
    cp_async16(smem_addr(w_s + row * RS + c8 * 8), src, in ? 16 : 0);
  }
  load_plane(z0 - 1);
  load_plane(z0);
  load_plane(z0 + 1);
  cp_async_commit();

  const int arow = lane & 15, ahalf = lane >> 4;  // A: row / k-half this lane addresses
  const int bm = lane >> 3, brow = lane & 7;      // B: matrix / row this lane addresses
  for (int z = z0; z < z1; ++z) {
    if (z + 2 <= z1) load_plane(z + 2);  // plane z1 is the last one the chunk reads
    cp_async_commit();                   // (possibly empty) group of plane z + 2
    cp_async_wait<1>();                  // everything but that group has landed: planes z-1 .. z+1
    __syncthreads();

    float acc[MT][NC / 8][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int t = 0; t < NC / 8; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][t][q] = 0.f;
    for (int tap = 0; tap < 27; ++tap) {
      const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
      const bf16* plane = ring + ((z - 1 + dz - (z0 - 1)) & 3) * SH::PLANE;
#pragma unroll
      for (int kc = 0; kc < CIN / 16; ++kc) {
        uint32_t af[MT][4];
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          const int tile = warp * MT + m;            // 2 tiles per output row
          const int row = tile >> 1, xh = (tile & 1) * 16;
          const bf16* ap = plane + ((row + dy) * PX + xh + arow + dx) * RS + ahalf * 8 + kc * 16;
          ldsm_x4(smem_addr(ap), af[m][0], af[m][1], af[m][2], af[m][3]);
        }
#pragma unroll
        for (int np = 0; np < NC / 16; ++np) {
          const int n = np * 16 + (bm >> 1) * 8 + brow;
          uint32_t b0, b1, b2, b3;
          ldsm_x4(smem_addr(w_s + (tap * NC + n) * RS + kc * 16 + (bm & 1) * 8), b0, b1, b2, b3);
#pragma unroll
          for (int m = 0; m < MT; ++m) {
            mma_bf16(acc[m][2 * np], af[m][0], af[m][1], af[m][2], af[m][3], b0, b1);
            mma_bf16(acc[m][2 * np + 1], af[m][0], af[m][1], af[m][2], af[m][3], b2, b3);
          }
        }
      }
    }
    // epilogue: bias, ReLU, bf16, split over the two outputs
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const int tile = warp * MT + m;
      const int gy = y0 + (tile >> 1);
      if (gy >= a.ny) continue;
#pragma unroll
      for (int t = 0; t < NC / 8; ++t) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int gx = x0 + (tile & 1) * 16 + (lane >> 2) + 8 * h;
          const int co = n0 + t * 8 + 2 * (lane & 3);
          if (gx >= a.nx || co >= a.cout) continue;
          float v0 = acc[m][t][2 * h], v1 = acc[m][t][2 * h + 1];
          if (a.bias) {
            v0 += a.bias[co];
            v1 += a.bias[co + 1];
          }
          if (a.relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          }
          const long long gv = gx + (long long)a.nx * (gy + (long long)a.ny * z);
          __nv_bfloat162 pv = __floats2bfloat162_rn(v0, v1);
          if (co < a.o1) *reinterpret_cast<__nv_bfloat162*>(a.out1 + gv * a.o1 + co) = pv;
          else *reinterpret_cast<__nv_bfloat162*>(a.out2 + gv * a.o2 + (co - a.o1)) = pv;
        }
      }
    }
    __syncthreads();  // plane z-1's slot is refilled (with plane z+3) in the next step
  }
  cp_async_wait<0>();  // no copy is left in flight when the CTA retires
}

// ------------------------------------------------------------------------------------------------
// The same 3x3x3 convolution on the 5th-generation tensor cores: tcgen05.mma with FP32 accumulators
// in TMEM, input planes staged by TMA (cp.async.bulk.tensor), warp-specialised and pipelined.
// A CTA owns an 8 x 16 tile of output voxels in (x, y) (M = 128 rows of the MMA, row m = voxel
// (x0 + m % 8, y0 + m / 8)), all NC output channels, and marches a chunk of z-planes.
// The MMAs are organised by input plane, not by output plane: staged plane p feeds output planes
// p+1, p and p-1 through the z-taps dz = 0, 1, 2, so for each in-plane tap (dy, dx) one MMA with the
// three z-taps' weights stacked along N (N = 3 NC) reads the plane's window once and adds to three
// accumulators.  The accumulators live in a ring of R blocks of NC TMEM columns, output plane j of the
// chunk in block R-1 - j % R: the blocks of outputs j, j-1, j-2 are adjacent in that order, so one MMA
// writes all three (two MMAs where the ring wraps, one or two blocks at the chunk's ends).  Every MMA
// accumulates; a block is zeroed (tcgen05.st) at the start and by the epilogue after it drains it.
//   warp 0 (lane 0): the producer.  Input plane p is staged once, with its halo, as
//     [g = CIN/8][r = 18 rows][v = 10 voxels] lines of 16 B (8 channels): one 5D TMA box
//     {8 channels, 1 group, 10 voxels, 18 rows, 1 plane} per channel group, zero-filled outside the
//     grid.  In the canonical K-major layout without swizzle a core matrix is 8 consecutive lines,
//     here the 8 voxels of one tile row; the tap (dy, dx) window starts at line dy * 10 + dx, its
//     16 core matrices along M (the tile's rows) are 10 lines = 160 B apart (SBO) and the channel
//     groups GROUP bytes apart (LBO).  The x shift of a tap is thus a start offset, not a copy.  A
//     ring of S planes; each plane is read by the MMAs of one step and then released.
//   warp 1 (lane 0): the MMA issuer.  For staged plane i of the chunk it issues 9 * CIN / 16 MMAs
//     (more where the ring wraps), then commits them to the plane's "empty" barrier and to the
//     "full" barrier of output i-2, which plane i completes.
//   warps 2..5: the epilogue.  Warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows 4 (w % 4) ..
//     +3) of a finished block, zeroes it and hands it back, then adds the bias, applies the ReLU and
//     stores bf16 (16 B per 8 channels) to the one or two outputs.
// Weights: [t = dy*3 + dx][g][n3 = dz * NC + n] lines (SBO 128 B, LBO 3 NC * 16 B), staged once per
// CTA with cp.async.  Every wait is bounded; a role that gives up records it in g_conv_timeout and
// raises the CTA's stop flag, the other roles leave their loops at their next wait, and the CTA frees
// its TMEM only after a bounded wait for its last MMAs.
// ------------------------------------------------------------------------------------------------
__device__ int g_conv_timeout;

template <int CIN, int NC, int S>
struct UmmaShape {
  static constexpr int TX = 8, TY = 16, PX = TX + 2, PY = TY + 2;  // tile and staged plane (with halo)
  static constexpr int LINES = PX * PY;                             // lines per channel group
  static constexpr int CG = CIN / 8;
  static constexpr int BOX = LINES * 16;                            // bytes one TMA box delivers
  static constexpr int GROUP = ((BOX + 127) / 128) * 128;           // bytes per group (128 B aligned boxes)
  static constexpr int PLANE = CG * GROUP;                          // bytes of a staged plane
  static constexpr int N3 = 3 * NC;                                 // the three z-taps' output channels
  static constexpr int WBYTES = 9 * CG * N3 * 16;
  static constexpr int OFF_RING = ((WBYTES + 1023) / 1024) * 1024;
  static constexpr int OFF_BAR = OFF_RING + S * PLANE;
  static constexpr int R = NC == 64 ? 4 : 8;                        // accumulator blocks in TMEM
  static constexpr int NBAR = 2 * S + 2 * R + 1;                    // full[S], empty[S], accf[R], acce[R], done
  static constexpr int OFF_BIAS = OFF_BAR + NBAR * 8 + 16;          // NC FP32 biases (zero past cout or without bias)
  static constexpr int TMEM_COLS = R * NC <= 32 ? 32 : (R * NC <= 64 ? 64 : (R * NC <= 128 ? 128 : 256));
  static constexpr int smem() { return OFF_BIAS + NC * 4 + 1024; }  // + slack for 1 KB alignment
};

__device__ inline uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);  // version 1, no swizzle, base offset 0
}
// kind::f16 instruction descriptor: D f32, A and B bf16, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ inline bool tc_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (each try_wait suspends for a while); stop != nullptr: also give up once another role
// of the CTA has raised the stop flag
__device__ inline bool tc_mbar_wait(uint32_t bar, uint32_t parity, const volatile int* stop = nullptr) {
  for (int it = 0; it < (1 << 22); ++it) {
    if (tc_try_wait(bar, parity)) return true;
    if (stop && (it & 63) == 63 && *stop) return false;
  }
  return false;
}
__device__ inline void tc_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ inline void tc_mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ inline void tc_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ inline void tc_tma_load_5d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3, int c4,
                                      uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}
__device__ inline void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ inline void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}
// zero 16 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ inline void tc_st16_zero(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}
// one MMA of M = 128 into TMEM columns dcol.., N = n (16 .. 256, a multiple of 16), accumulating
__device__ inline void tc_mma_acc(uint32_t dcol, uint64_t ad, uint64_t bd, int n) {
  const uint32_t idesc = tc_idesc_bf16(128, 0) | ((uint32_t)(n >> 3) << 17);
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
      "l"(ad), "l"(bd), "r"(idesc), "r"(1u)
      : "memory");
}

// tm1 / tm2: 5D maps {8 channels, groups, nx, ny, nz} of the two inputs (box {8, 1, 10, 18, 1});
// tm2 is unused when a.c2 == 0.  Every channel count a multiple of 8; with cout > NC the output
// channels are split into blocks of NC over blockIdx.z.
template <int CIN, int NC, int S>
__global__ void __launch_bounds__(192) conv3_tc_kernel(const __grid_constant__ CUtensorMap tm1,
                                                       const __grid_constant__ CUtensorMap tm2, ConvArgs a, int tz) {
  using SH = UmmaShape<CIN, NC, S>;
  constexpr int CG = SH::CG, R = SH::R, N3 = SH::N3;
  static_assert(CIN % 16 == 0 && NC % 16 == 0 && NC <= 64 && N3 <= 256 && S >= 2 && SH::smem() <= 232448,
                "tcgen05 conv shape");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t w_s = smem_addr(smem), ring = smem_addr(smem + SH::OFF_RING);
  const uint32_t bar0 = smem_addr(smem + SH::OFF_BAR);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (S + s); };
  auto accf = [&](int r) { return bar0 + 8u * (2 * S + r); };
  auto acce = [&](int r) { return bar0 + 8u * (2 * S + R + r); };
  const uint32_t done = bar0 + 8u * (2 * S + 2 * R);
  uint32_t* tmem_slot = (uint32_t*)(smem + SH::OFF_BAR + SH::NBAR * 8);
  volatile int* stop = (volatile int*)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * SH::TX, y0 = blockIdx.y * SH::TY;
  // blockIdx.z = z-chunk * nblk + output-channel block: a CTA computes output channels n0 .. n0+NC-1
  const int nblk = (a.cout + NC - 1) / NC, n0 = (blockIdx.z % nblk) * NC;
  const int z0 = (blockIdx.z / nblk) * tz, z1 = min(a.nz, z0 + tz);
  if (z0 >= z1) return;  // uniform over the CTA, before any TMEM is taken
  const int nout = z1 - z0, nplanes = nout + 2;  // planes z0-1 .. z1
  const int cg1 = a.c1 / 8, cg2 = a.c2 / 8;

  if (warp == 1) {  // TMEM: R accumulator blocks of NC FP32 columns (128 lanes)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "n"(SH::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc_mbar_init(full(s), 1);
      tc_mbar_init(empty(s), 1);
    }
    for (int r = 0; r < R; ++r) {
      tc_mbar_init(accf(r), 1);
      tc_mbar_init(acce(r), 4);
    }
    tc_mbar_init(done, 1);
    *stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights: line (t, g, dz * NC + n) = W[dz * 9 + t][n0 + n][8g .. 8g+7] (channels beyond cout are zero)
  for (int q = tid; q < 9 * CG * N3; q += 192) {
    const int n3 = q % N3, g = (q / N3) % CG, t = q / (N3 * CG);
    const int dz = n3 / NC, n = n3 % NC;
    const bool in = n0 + n < a.cout;
    const void* src =
        in ? (const void*)(a.w + ((long long)(dz * 9 + t) * a.cout + n0 + n) * CIN + g * 8) : (const void*)a.w;
    cp_async16(w_s + q * 16, src, in ? 16 : 0);
  }
  cp_async_commit();
  float* bias_s = (float*)(smem + SH::OFF_BIAS);
  for (int n = tid; n < NC; n += 192) bias_s[n] = (a.bias && n0 + n < a.cout) ? a.bias[n0 + n] : 0.f;
  cp_async_wait<0>();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the weights, to the tensor core's reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (warp >= 2) {  // every accumulator block starts at zero (all MMAs accumulate)
    const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
    for (int c = 0; c < R * NC; c += 16) tc_st16_zero(tl + c);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  auto fail = [&]() {
    atomicExch(&g_conv_timeout, 1);
    *stop = 1;
  };
  auto blk = [&](int j) { return (R - 1) - j % R; };  // the TMEM block of output plane j of the chunk

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int i = 0;
      for (; i < nplanes; ++i) {
        const int s = i % S;
        if (i >= S && !tc_mbar_wait(empty(s), ((i / S) - 1) & 1, stop)) {
          fail();
          break;
        }
        const int p = z0 - 1 + i;
        const uint32_t dst = ring + s * SH::PLANE;
        tc_expect_tx(full(s), CG * SH::BOX);  // the boxes' bytes (the 64 B of padding per group stay unwritten)
        for (int g = 0; g < cg1; ++g) tc_tma_load_5d(dst + g * SH::GROUP, &tm1, 0, g, x0 - 1, y0 - 1, p, full(s));
        for (int g = 0; g < cg2; ++g)
          tc_tma_load_5d(dst + (cg1 + g) * SH::GROUP, &tm2, 0, g, x0 - 1, y0 - 1, p, full(s));
      }
      // every copy issued lands before the CTA retires (the last S issued; earlier ones were consumed)
      for (int d = 1; d <= S && d <= i; ++d) (void)tc_mbar_wait(full((i - d) % S), ((i - d) / S) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint64_t bdesc = tc_smem_desc(w_s, N3 * 16, 128);
      for (int i = 0; i < nplanes; ++i) {
        // plane i feeds outputs j = i - dz for dz in [dz_lo, dz_hi] (those inside the chunk)
        const int dz_lo = max(0, i - (nout - 1)), dz_hi = min(2, i);
        bool ok = tc_mbar_wait(full(i % S), (i / S) & 1, stop);
        if (ok && dz_lo == 0 && i >= R) ok = tc_mbar_wait(acce(i % R), ((i / R) - 1) & 1, stop);  // block of output i free
        if (!ok) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the dz range in at most two runs of adjacent blocks: the ring wraps after the output whose
        // block is R-1 (j % R == 0), at most once in three outputs (R >= 4)
        int brk = -1;
        for (int dz = dz_lo; dz < dz_hi; ++dz)
          if ((i - dz) % R == 0) brk = dz;
        const int a1 = dz_lo, b1 = brk >= 0 ? brk : dz_hi;  // first run
        const int a2 = b1 + 1;                                // second run: a2 .. dz_hi when brk >= 0
        const uint64_t adesc = tc_smem_desc(ring + (i % S) * SH::PLANE, SH::GROUP, SH::PX * 16);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const int dy = t / 3, dx = t % 3;
#pragma unroll
          for (int kk = 0; kk < CIN / 16; ++kk) {
            const uint64_t ad = adesc + (uint64_t)(((dy * SH::PX + dx) * 16 + kk * 2 * SH::GROUP) >> 4);
            const uint64_t bt = bdesc + (uint64_t)(((t * CG + 2 * kk) * N3 * 16) >> 4);
            tc_mma_acc(tmem + (uint32_t)(blk(i - a1) * NC), ad, bt + (uint64_t)((a1 * NC * 16) >> 4), (b1 - a1 + 1) * NC);
            if (brk >= 0)
              tc_mma_acc(tmem + (uint32_t)(blk(i - a2) * NC), ad, bt + (uint64_t)((a2 * NC * 16) >> 4),
                         (dz_hi - a2 + 1) * NC);
          }
        }
        tc_commit(empty(i % S));                   // plane i is no longer read
        if (dz_hi == 2) tc_commit(accf((i - 2) % R));  // output i-2 has all its contributions
      }
      tc_commit(done);  // every MMA this CTA issued has completed once this barrier flips
      (void)tc_mbar_wait(done, 0);
    }
  } else {
    // ---------------- epilogue: warps 2..5 ----------------
    const int q = warp & 3;  // TMEM lanes 32q .. 32q+31 = tile rows 4q .. 4q+3
    const int gx = x0 + (lane & 7), gy = y0 + 4 * q + (lane >> 3);
    const bool valid = gx < a.nx && gy < a.ny;
    for (int j = 0; j < nout; ++j) {
      const bool ok = __all_sync(0xffffffffu, tc_mbar_wait(accf(j % R), (j / R) & 1, stop));
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float v[NC];
      const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(blk(j) * NC);
#pragma unroll
      for (int h = 0; h < NC / 16; ++h) tc_ld16(taddr + 16 * h, v + 16 * h);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int h = 0; h < NC / 16; ++h) tc_st16_zero(taddr + 16 * h);  // the block's next output starts at zero
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) tc_mbar_arrive(acce(j % R));  // the block may take output j + R
      if (valid) {
        const long long gv = gx + (long long)a.nx * (gy + (long long)a.ny * (z0 + j));
#pragma unroll
        for (int c8 = 0; c8 < NC / 8; ++c8) {
          const int cl = c8 * 8, co = n0 + cl;  // the block's channel and the layer's
          if (co >= a.cout) break;
          uint32_t pk[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float v0 = v[cl + 2 * e] + bias_s[cl + 2 * e], v1 = v[cl + 2 * e + 1] + bias_s[cl + 2 * e + 1];
            if (a.relu) {
              v0 = fmaxf(v0, 0.f);
              v1 = fmaxf(v1, 0.f);
            }
            const __nv_bfloat162 pv = __floats2bfloat162_rn(v0, v1);
            pk[e] = *reinterpret_cast<const uint32_t*>(&pv);
          }
          bf16* dst = co < a.o1 ? a.out1 + gv * a.o1 + co : a.out2 + gv * a.o2 + (co - a.o1);
          *reinterpret_cast<uint4*>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(SH::TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------------------------------------------
// Weight gradient of a 3x3x3 convolution:
//   dW[tap][co][ci] += sum_v dy[v][co] * x[v + off(tap)][ci],   db[co] += sum_v dy[v][co]
// ------------------------------------------------------------------------------------------------
struct WgradArgs {
  const bf16* dy;  // [N][cout]
  const bf16* x1;
  const bf16* x2;
  int c1, c2;      // input channels of the forward conv (split over two sources)
  int cout;
  float* dw;       // [27][cout][c1 + c2]
  float* db;       // [cout] or null (accumulated by tap 13)
  int nx, ny, nz;
  int chunk;       // voxels per CTA
};

// On the tensor cores (mma.sync m16n8k16, bf16 x bf16 -> FP32): for one tap,
//   dW[tap] (CO x CI) += dY^T (CO x V) X_tap (V x CI),   X_tap[v] = x[v + off(tap)] (zero outside),
// a GEMM whose K dimension is the voxels.  A block takes one tap (blockIdx.y) and a chunk of voxels
// (blockIdx.x), stages 64 voxels at a time as [voxel][channel] rows of dY and of the shifted X (rows
// padded by 8 channels, so that the 8 rows an ldmatrix reads start in distinct banks) and reads them as
// transposed fragments (ldmatrix .trans): the MMA's A operand is dY^T, its B operand X_tap.  The 4 K-steps
// of 16 voxels times the (CO/16) x (CI/8) output tiles are spread over the 8 warps, each warp keeping
// FP32 accumulators for its tiles across all of the block's voxels; the block's partial dW is added with
// FP32 atomics, and the centre tap's blocks also sum dY for db.
// ------------------------------------------------------------------------------------------------
__device__ inline void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ inline void ldsm_x2_t(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

template <int CO, int CI>
__global__ void __launch_bounds__(256) conv3_wgrad_mma_kernel(WgradArgs a) {
  constexpr int TV = 64, RSO = CO + 8, RSI = CI + 8;
  constexpr int MT = CO / 16, NT = CI / 8, TILES = MT * NT;
  constexpr int NACC = TILES >= 8 ? TILES / 8 : 1;  // output tiles per warp
  static_assert(CO % 16 == 0 && CI % 8 == 0 && (TILES % 8 == 0 || 8 % TILES == 0), "wgrad tile shape");
  __shared__ __align__(16) bf16 sdy[TV * RSO];
  __shared__ __align__(16) bf16 sx[TV * RSI];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tap = blockIdx.y;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const long long nvox = (long long)a.nx * a.ny * a.nz;
  const long long v0 = (long long)blockIdx.x * a.chunk;
  const long long v1 = min(nvox, v0 + a.chunk);
  float acc[NACC][4];
#pragma unroll
  for (int j = 0; j < NACC; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  float dbs = 0.f;
  const int q = lane >> 3, r = lane & 7;  // ldmatrix: which 8x8 matrix this lane addresses, and its row
  for (long long vb = v0; vb < v1; vb += TV) {
    __syncthreads();  // the previous tile's fragments are read
    for (int e = tid; e < TV * (CO / 8); e += 256) {  // dY rows, 16-byte vectors
      const int vi = e / (CO / 8), c8 = e % (CO / 8);
      const long long v = vb + vi;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (v < v1) val = *reinterpret_cast<const uint4*>(a.dy + v * CO + c8 * 8);
      *reinterpret_cast<uint4*>(sdy + vi * RSO + c8 * 8) = val;
    }
    for (int e = tid; e < TV * (CI / 8); e += 256) {  // X rows shifted by the tap
      const int vi = e / (CI / 8), c8 = e % (CI / 8);
      const long long v = vb + vi;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (v < v1) {
        const int x = (int)(v % a.nx), y = (int)((v / a.nx) % a.ny), z = (int)(v / ((long long)a.nx * a.ny));
        const int xs = x + dx, ys = y + dy, zs = z + dz;
        if (xs >= 0 && ys >= 0 && zs >= 0 && xs < a.nx && ys < a.ny && zs < a.nz) {
          const long long vs = xs + (long long)a.nx * (ys + (long long)a.ny * zs);
          const int c = c8 * 8;
          val = c < a.c1 ? *reinterpret_cast<const uint4*>(a.x1 + vs * a.c1 + c)
                         : *reinterpret_cast<const uint4*>(a.x2 + vs * a.c2 + (c - a.c1));
        }
      }
      *reinterpret_cast<uint4*>(sx + vi * RSI + c8 * 8) = val;
    }
    __syncthreads();
    if (a.db && tap == 13 && tid < CO)
      for (int vi = 0; vi < TV; ++vi) dbs += __bfloat162float(sdy[vi * RSO + tid]);
#pragma unroll
    for (int j = 0; j < NACC; ++j) {
      const int tile = TILES >= 8 ? warp + 8 * j : warp % TILES;
      const int mt = tile / NT, nt = tile % NT;
      // K-steps of this warp for this tile: all four, or (with fewer tiles than warps) every 8/TILES-th
      constexpr int KSTEP = TILES >= 8 ? 1 : 8 / TILES;
      const int k_first = TILES >= 8 ? 0 : warp / TILES;
#pragma unroll
      for (int ks = k_first; ks < TV / 16; ks += KSTEP) {
        const int kk = ks * 16;
        uint32_t a0, a1, a2, a3, b0, b1;
        ldsm_x4_t(smem_addr(sdy + (kk + (q >> 1) * 8 + r) * RSO + mt * 16 + (q & 1) * 8), a0, a1, a2, a3);
        ldsm_x2_t(smem_addr(sx + (kk + (lane & 15)) * RSI + nt * 8), b0, b1);
        mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
      }
    }
  }
  const int cin = a.c1 + a.c2;
#pragma unroll
  for (int j = 0; j < NACC; ++j) {
    const int tile = TILES >= 8 ? warp + 8 * j : warp % TILES;
    const int mt = tile / NT, nt = tile % NT;
    const int m = mt * 16 + (lane >> 2), n = nt * 8 + 2 * (lane & 3);
    float* w0 = a.dw + ((long long)tap * CO + m) * cin + n;
    atomicAdd(w0, acc[j][0]);
    atomicAdd(w0 + 1, acc[j][1]);
    atomicAdd(w0 + 8LL * cin, acc[j][2]);
    atomicAdd(w0 + 8LL * cin + 1, acc[j][3]);
  }
  if (a.db && tap == 13 && tid < CO) atomicAdd(&a.db[tid], dbs);
}

// ---- pooling ------------------------------------------------------------------------------------
// out (coarse, n/2 per axis) = mean of the 8 children; backward: each child gets dout / 8
__global__ void pool_fwd_kernel(const bf16* in, bf16* out, int c, int nx, int ny, int nz) {
  // one thread per (coarse voxel, group of 8 channels): eight 16-byte loads, one 16-byte store
  const int mx = nx / 2, my = ny / 2, mz = nz / 2, g8 = c / 8;
  const int n = mx * my * mz * g8;  // below 2^31 for any grid that fits
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int cg = t % g8, V = t / g8;
  const int X = V % mx, Y = (V / mx) % my, Z = V / (mx * my);
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int x = 2 * X + (q & 1), y = 2 * Y + ((q >> 1) & 1), z = 2 * Z + (q >> 2);
    const uint4 u = *reinterpret_cast<const uint4*>(in + (x + (long long)nx * (y + (long long)ny * z)) * c + cg * 8);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(h[e]);
      s[2 * e] += f.x;
      s[2 * e + 1] += f.y;
    }
  }
  uint4 u;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(0.125f * s[2 * e], 0.125f * s[2 * e + 1]);
  *reinterpret_cast<uint4*>(out + (long long)V * c + cg * 8) = u;
}

__global__ void pool_bwd_kernel(const bf16* dout, bf16* din, int c, int nx, int ny, int nz) {
  const long long n = (long long)nx * ny * nz * c;
  const int mx = nx / 2, my = ny / 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(t % c);
    const long long v = t / c;
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
    const long long V = (x / 2) + (long long)mx * ((y / 2) + (long long)my * (z / 2));
    din[t] = __float2bfloat16(0.125f * __bfloat162float(dout[V * c + ch]));
  }
}

// ---- 2x2x2 transposed convolution, stride 2 (coarse -> fine) -------------------------------------
// out[x][y][z][co] = b[co] + sum_ci in[x/2][y/2][z/2][ci] * W[(z%2, y%2, x%2)][co][ci], W rounded to
// bf16 (like the 3x3x3 convolutions' weights), b in FP32
template <int CIN, int COUT>
constexpr int tconv_smem() {
  return (COUT * CIN * 8 + COUT) * (int)sizeof(float);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(256) tconv_fwd_kernel(const bf16* in, const float* w, const float* b, bf16* out,
                                                        int mx, int my, int mz) {
  // one thread per (coarse voxel V, child k = kx + 2 ky + 4 kz), k fastest; the weights are staged
  // as [co][ci][k] so that the 8 children in a warp read 8 banks and its 4 voxels share them
  extern __shared__ float tc_smem[];  // COUT * CIN * 8 weights, then COUT biases (tconv_smem<CIN, COUT>)
  float* w_s = tc_smem;
  float* b_s = tc_smem + COUT * CIN * 8;
  for (int q = threadIdx.x; q < COUT * CIN * 8; q += blockDim.x) {
    const int k = q & 7, ci = (q >> 3) % CIN, co = (q >> 3) / CIN;
    w_s[q] = __bfloat162float(__float2bfloat16(w[(k * COUT + co) * CIN + ci]));
  }
  for (int q = threadIdx.x; q < COUT; q += blockDim.x) b_s[q] = b[q];
  __syncthreads();
  const int nvc = mx * my * mz;  // coarse voxels (below 2^31 / 8 for any grid that fits)
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8 * nvc) return;
  const int k = t & 7, V = t >> 3;
  const int x = V % mx, y = (V / mx) % my, z = V / (mx * my);
  const int X = 2 * x + (k & 1), Y = 2 * y + ((k >> 1) & 1), Z = 2 * z + (k >> 2);
  const long long child = X + 2LL * mx * (Y + 2LL * my * Z);
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = b_s[co];
  const uint4* ip = reinterpret_cast<const uint4*>(in + (long long)V * CIN);
#pragma unroll
  for (int c8 = 0; c8 < CIN / 8; ++c8) {
    const uint4 u = ip[c8];
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(h[e]);
      const int ci = c8 * 8 + 2 * e;
#pragma unroll
      for (int co = 0; co < COUT; ++co) {
        acc[co] = fmaf(f.x, w_s[(co * CIN + ci) * 8 + k], acc[co]);
        acc[co] = fmaf(f.y, w_s[(co * CIN + ci + 1) * 8 + k], acc[co]);
      }
    }
  }
  uint4* op = reinterpret_cast<uint4*>(out + child * COUT);
#pragma unroll
  for (int c8 = 0; c8 < COUT / 8; ++c8) {
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(acc[c8 * 8 + 2 * e], acc[c8 * 8 + 2 * e + 1]);
    op[c8] = u;
  }
}

// The same transposed convolution on the 5th-generation tensor cores, one GEMM per tile of 128
// consecutive coarse voxels V0 .. V0+127:
//   D[V][k * COUT + co] = sum_ci in[V][ci] * W[k][co][ci]      (M = 128, N = 8 * COUT, K = CIN)
//   out[child(V, k)][co] = bf16(D[V][k * COUT + co] + b[co])
// with bf16 weights (rounded from the FP32 master copy when the CTA stages them) and FP32
// accumulation in TMEM.  Operands in the canonical K-major layout without swizzle: the tile as
// [g = CIN/8][v = 128] lines of 16 B (cp.async, zero fill past the last voxel), the weights as
// [g][n = 8 * COUT] lines.  Persistent CTAs of 4 warps (warp w reads TMEM lanes 32w .. 32w+31, one
// coarse voxel per thread); the dynamic shared memory is padded so that no more CTAs share an SM
// than its 512 TMEM columns hold.
template <int CIN, int COUT>
struct TconvTc {
  static constexpr int CG = CIN / 8, N = 8 * COUT;
  static constexpr int ABYTES = CG * 128 * 16;
  static constexpr int BBYTES = CG * N * 16;
  static constexpr int OFF_BAR = ABYTES + BBYTES;
  static constexpr int PER_SM = 512 / N;  // CTAs whose accumulators fit in one SM's TMEM
  static constexpr int need() { return OFF_BAR + 32 + 1024; }  // two barriers, the TMEM address, alignment slack
  static constexpr int smem() {
    return need() > 232448 / (PER_SM + 1) + 1024 ? need() : 232448 / (PER_SM + 1) + 1024;
  }
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128) tconv_tc_kernel(const bf16* in, const float* w, const float* b, bf16* out,
                                                       int mx, int my, int mz) {
  using SH = TconvTc<CIN, COUT>;
  constexpr int CG = SH::CG, N = SH::N;
  static_assert(CIN % 16 == 0 && COUT % 16 == 0 && N <= 256, "tcgen05 transposed conv shape");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t a_s = smem_addr(smem), b_s = smem_addr(smem + SH::ABYTES);
  const uint32_t bar = smem_addr(smem + SH::OFF_BAR), done = bar + 8;
  uint32_t* tmem_slot = (uint32_t*)(smem + SH::OFF_BAR + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long nvc = (long long)mx * my * mz;
  const long long ntiles = (nvc + 127) / 128;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "n"(N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    tc_mbar_init(bar, 1);
    tc_mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights: line (g, n = k * COUT + co) holds bf16(W[k][co][8g .. 8g+7])
  for (int q = tid; q < CG * N; q += 128) {
    const int n = q % N, g = q / N;
    const float* src = w + (long long)n * CIN + g * 8;
    uint32_t pk[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat162 pv = __floats2bfloat162_rn(src[2 * e], src[2 * e + 1]);
      pk[e] = *reinterpret_cast<const uint32_t*>(&pv);
    }
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(b_s + q * 16), "r"(pk[0]), "r"(pk[1]), "r"(pk[2]),
                 "r"(pk[3])
                 : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
  constexpr uint32_t IDESC = tc_idesc_bf16(128, N);

  int it = 0;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const long long V0 = t * 128;
    for (int q = tid; q < 128 * CG; q += 128) {  // line (g, v) <- in[V0 + v][8g .. 8g+7]
      const int v = q % 128, g = q / 128;
      const bool ok = V0 + v < nvc;
      cp_async16(a_s + (g * 128 + v) * 16, ok ? (const void*)(in + (V0 + v) * CIN + g * 8) : (const void*)in, ok ? 16 : 0);
    }
    cp_async_commit();
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the tile and the weights, to the tensor core
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < CIN / 16; ++kk) {
        const uint64_t ad = tc_smem_desc(a_s + kk * 2 * 128 * 16, 128 * 16, 128);
        const uint64_t bd = tc_smem_desc(b_s + kk * 2 * N * 16, N * 16, 128);
        const uint32_t acc = kk != 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
            : "memory");
      }
      tc_commit(bar);
    }
    const bool ok = tc_mbar_wait(bar, it & 1);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(&g_conv_timeout, 1);
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const long long V = V0 + 32 * warp + lane;
    const bool valid = V < nvc;
    const int x = (int)(V % mx), y = (int)((V / mx) % my), z = (int)(V / ((long long)mx * my));
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
      float v[COUT];
#pragma unroll
      for (int h = 0; h < COUT / 16; ++h) tc_ld16(taddr + k * COUT + 16 * h, v + 16 * h);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (!valid) continue;
      const long long child =
          (2 * x + (k & 1)) + 2LL * mx * ((2 * y + ((k >> 1) & 1)) + 2LL * my * (2 * z + (k >> 2)));
      uint4* op = reinterpret_cast<uint4*>(out + child * COUT);
#pragma unroll
      for (int c8 = 0; c8 < COUT / 8; ++c8) {
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int co = c8 * 8 + 2 * e;
          const __nv_bfloat162 pv = __floats2bfloat162_rn(v[co] + b[co], v[co + 1] + b[co + 1]);
          pk[e] = *reinterpret_cast<const uint32_t*>(&pv);
        }
        op[c8] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // TMEM read out and the tile's smem free before the next tile
  }
  if (tid == 0) {  // every MMA issued has completed before the columns are freed (bounded)
    tc_commit(done);
    (void)tc_mbar_wait(done, 0);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(N) : "memory");
  }
}

// din[V][ci] = sum_{k, co} dout[child(V, k)][co] * W[k][co][ci]
__global__ void tconv_bwd_data_kernel(const bf16* dout, const float* w, bf16* din, int cin, int cout, int nx, int ny,
                                      int nz) {
  const int mx = nx / 2, my = ny / 2, mz = nz / 2;
  const long long n = (long long)mx * my * mz * cin;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(t % cin);
    const long long V = t / cin;
    const int X = (int)(V % mx), Y = (int)((V / mx) % my), Z = (int)(V / ((long long)mx * my));
    float s = 0.f;
    for (int k = 0; k < 8; ++k) {
      const int x = 2 * X + (k & 1), y = 2 * Y + ((k >> 1) & 1), z = 2 * Z + (k >> 2);
      const bf16* dp = dout + (x + (long long)nx * (y + (long long)ny * z)) * cout;
      const float* wp = w + (long long)k * cout * cin + ci;
      for (int co = 0; co < cout; ++co)  // the bf16 weights the forward pass multiplies with
        s += __bfloat162float(dp[co]) * __bfloat162float(__float2bfloat16(wp[(long long)co * cin]));
    }
    din[t] = __float2bfloat16(s);
  }
}

// dW[k][co][ci] += sum_V in[V][ci] * dout[child(V, k)][co];  db[co] += sum dout[.][co]
// grid (coarse-voxel chunks, 8 children); one thread per (co, ci) pair (cout * cin <= 2048)
__global__ void tconv_bwd_weight_kernel(const bf16* in, const bf16* dout, float* dw, float* db, int cin, int cout,
                                        int nx, int ny, int nz, int chunk) {
  const int mx = nx / 2, my = ny / 2, mz = nz / 2;
  const long long nv = (long long)mx * my * mz;
  const int k = blockIdx.y;
  const long long V0 = (long long)blockIdx.x * chunk, V1 = min(nv, V0 + chunk);
  for (int pair = threadIdx.x; pair < cin * cout; pair += blockDim.x) {
    const int co = pair / cin, ci = pair % cin;
    float s = 0.f, sb = 0.f;
    for (long long V = V0; V < V1; ++V) {
      const int X = (int)(V % mx), Y = (int)((V / mx) % my), Z = (int)(V / ((long long)mx * my));
      const int x = 2 * X + (k & 1), y = 2 * Y + ((k >> 1) & 1), z = 2 * Z + (k >> 2);
      const float d = __bfloat162float(dout[(x + (long long)nx * (y + (long long)ny * z)) * cout + co]);
      s += __bfloat162float(in[V * cin + ci]) * d;
      sb += d;
    }
    atomicAdd(&dw[((long long)k * cout + co) * cin + ci], s);
    if (ci == 0) atomicAdd(&db[co], sb);
  }
}

// ---- 1x1x1 head (16 -> 6 channels, FP32 output) ----------------------------------------------------
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) head_fwd_kernel(const bf16* in, const float* w, const float* b, float* out,
                                                       int nv) {
  // one thread per voxel: its CIN channels in 16-byte loads, all COUT outputs
  __shared__ float w_s[COUT * CIN], b_s[COUT];
  for (int q = threadIdx.x; q < COUT * CIN; q += blockDim.x) w_s[q] = w[q];
  for (int q = threadIdx.x; q < COUT; q += blockDim.x) b_s[q] = b[q];
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = b_s[o];
  const uint4* ip = reinterpret_cast<const uint4*>(in + (long long)v * CIN);
#pragma unroll
  for (int c8 = 0; c8 < CIN / 8; ++c8) {
    const uint4 u = ip[c8];
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(h[e]);
#pragma unroll
      for (int o = 0; o < COUT; ++o)
        acc[o] = fmaf(f.y, w_s[o * CIN + c8 * 8 + 2 * e + 1], fmaf(f.x, w_s[o * CIN + c8 * 8 + 2 * e], acc[o]));
    }
  }
  float* op = out + (long long)v * COUT;
#pragma unroll
  for (int o = 0; o < COUT; ++o) op[o] = acc[o];
}

// din[v][c] = sum_o dout[v][o] W[o][c];  dW[o][c] += sum_v dout[v][o] in[v][c];  db[o] += sum_v dout[v][o]
__global__ void head_bwd_data_kernel(const float* dout, const float* w, bf16* din, int cin, int cout, long long nv) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nv * cin; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t % cin);
    const long long v = t / cin;
    float s = 0.f;
    for (int o = 0; o < cout; ++o) s += dout[v * cout + o] * w[o * cin + c];
    din[t] = __float2bfloat16(s);
  }
}

__global__ void __launch_bounds__(256) head_bwd_weight_kernel(const bf16* in, const float* dout, float* dw, float* db,
                                                              int cin, int cout, long long nv) {
  // one thread per (o, c) pair plus the bias; one block per chunk of 256 voxels
  const long long v0 = (long long)blockIdx.x * 256, v1 = min(nv, v0 + 256);
  for (int pair = threadIdx.x; pair < cout * (cin + 1); pair += blockDim.x) {
    const int o = pair / (cin + 1), c = pair % (cin + 1);
    float s = 0.f;
    for (long long v = v0; v < v1; ++v) {
      const float d = dout[v * cout + o];
      s += c < cin ? d * __bfloat162float(in[v * cin + c]) : d;
    }
    if (c < cin) atomicAdd(&dw[o * cin + c], s);
    else atomicAdd(&db[o], s);
  }
}

// a += b (bf16), for gradients that meet at a skip connection
__global__ void bf16_add_kernel(bf16* a, const bf16* b, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    a[t] = __float2bfloat16(__bfloat162float(a[t]) + __bfloat162float(b[t]));
}

// g = g * (y > 0)   (ReLU backward on the stored post-activation y)
__global__ void relu_bwd_kernel(bf16* g, const bf16* y, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(y[t]) > 0.f)) g[t] = __float2bfloat16(0.f);
}

// ---- loss: L = ||y - t||^2 / ||t||^2 over a sample, dy = 2 (y - t) / ||t||^2 -----------------------
__global__ void loss_sums_kernel(const float* y, const float* t, long long n, double* sums) {
  double a = 0.0, b = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double d = (double)y[i] - (double)t[i];
    a += d * d;
    b += (double)t[i] * (double)t[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], b);
  }
}

__global__ void loss_grad_kernel(const float* y, const float* t, long long n, const double* sums, float* dy) {
  // a zero target (an iterate that already is the solution) carries no direction: no gradient
  const float sc = sums[1] > 1e-30 ? (float)(2.0 / sums[1]) : 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dy[i] = sc * (y[i] - t[i]);
}

// ---- Adam on the flat FP32 master parameters ---------------------------------------------------
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// forward copy W[tap][co][ci] -> bf16, and the dgrad copy Wt[26 - tap][ci][co]
__global__ void conv_weights_bf16_kernel(const float* w, bf16* wf, bf16* wt, int cout, int cin) {
  const long long n = 27LL * cout * cin;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(t % cin), co = (int)((t / cin) % cout), tap = (int)(t / ((long long)cin * cout));
    const bf16 b = __float2bfloat16(w[t]);
    wf[t] = b;
    wt[((long long)(26 - tap) * cin + ci) * cout + co] = b;
  }
}

// deterministic counter-based normal draws for weight initialisation (splitmix64 + Box-Muller)
__device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}
__global__ void init_normal_kernel(float* p, long long n, float stdv, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed ^ (2 * (uint64_t)i)), b = splitmix64(seed ^ (2 * (uint64_t)i + 1));
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0), u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    p[i] = (float)(stdv * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
  }
}

}  // namespace unet
