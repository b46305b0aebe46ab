// Fused TMA-staged stencil apply for sm_103a: one kernel, one pass over HBM.
//
// Computes the same operator as the generic kernel in fit_stencil.cu (Eq. e2 with the Eq. CP
// curl, matrix-free as in Sec. III / Eq. e2t but fused: h = M_nu C e lives only in registers):
//     y = out_scale * [ C^T M_nu C (P x) - w^2 M_eps x + j w M_kappa x ],   y = x on masked edges.
//
// Decomposition.  A CTA owns a tile of TX x TY cells in the (x, y) plane and a chunk of TZ planes
// along z; one thread owns one (i, j) column and marches up the chunk.  For every plane the CTA
// stages, with bulk tensor copies (cp.async.bulk.tensor, TMA) into a ring of S shared-memory
// stages completed on mbarriers:
//     e     (TX+4) x (TY+2) cells x 3 complex   (x from i0-2 so the copy starts 16-byte aligned)
//     M_nu  (TX+4) x (TY+1) cells x 3           (x from i0-4, the same alignment rule)
//     M_eps, M_kappa  TX x TY cells x 6         (own cells only)
//     mask  (TX+32) x (TY+2) bytes              (x from i0-16)
// Out-of-grid boxes are zero-filled by the copy engine, which is exactly the truncation of the
// forward differences at the walls.  After a plane lands, masked edges of the staged e are zeroed
// (the P in P C^T M_nu C P).  At plane k a thread needs e at planes k and k+1 and h at plane k-1 of
// its own column, which it carries in registers from the previous step, together with e of its
// own, its x-1 and its y-1 cell.  The output plane of the tile is staged in shared memory (two
// buffers) and written with a bulk tensor store; CTAs are persistent (one wave) and loop over tiles.
//
// Two kernels share this staging.  fused_apply_kernel is CTA-synchronous: thread 0 issues the
// copies, all warps mask a landed plane together, and CTA barriers separate the steps.
// ws_apply_kernel is warp-specialised (roles described above it): the copy-issuing warp refills a
// stage the moment the consumers release it, and consumers release a plane as soon as they have
// read it, so more of the ring is in flight at any time.  Either kernel may also request planes
// a few steps ahead into L2 (bulk tensor prefetch), decoupling DRAM latency from the ring depth.
// The autotuner picks the kernel, tile height, chunk length, ring depth and prefetch distance.
//
// Fused epilogues (fit_epi): <u, y>, <y, x> and <y, y>, or y = u - A x with <y, y>, accumulated
// per thread in the vector precision and reduced by fit_block_sum (FP64 from the warp level up).
//
// Every wait on an mbarrier is bounded; on timeout the CTA records an error code in the grid's
// device error word, waits (bounded) for the copies it issued, and returns.
#include <cuda.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "fit_internal.cuh"

namespace {

constexpr int TX = 32;  // one warp per tile row

template <typename T, int TY, bool KU = false>  // KU: the stage also holds the epilogue vector u
struct Layout {
  using V = typename cplx<T>::t;
  static constexpr int CE = sizeof(V) / 8;      // 8-byte copy elements per complex value
  static constexpr int EW = 3 * (TX + 4);       // complex values per staged e row
  static constexpr int ER = TY + 2;
  static constexpr int NW = 3 * (TX + 4);       // T values per staged M_nu row
  static constexpr int NR = TY + 1;
  static constexpr int KW = 6 * TX;             // T values per staged M_eps/M_kappa row
  static constexpr int MW = TX + 32;            // mask bytes per staged row
  static constexpr int MR = TY + 2;
  static constexpr int OW = 3 * TX;             // complex values per output / u row
  static constexpr int al(int b) { return (b + 127) / 128 * 128; }
  static constexpr int E_BYTES = EW * ER * (int)sizeof(V);
  static constexpr int N_BYTES = NW * NR * (int)sizeof(T);
  static constexpr int K_BYTES = KW * TY * (int)sizeof(T);
  static constexpr int M_BYTES = MW * MR;
  static constexpr int U_BYTES = OW * TY * (int)sizeof(V);  // also the size of one output buffer
  static constexpr int E_OFF = 0;
  static constexpr int N_OFF = al(E_BYTES);
  static constexpr int K_OFF = N_OFF + al(N_BYTES);
  static constexpr int M_OFF = K_OFF + al(K_BYTES);
  static constexpr int U_OFF = M_OFF + al(M_BYTES);
  static constexpr int STAGE = U_OFF + (KU ? al(U_BYTES) : 0);
  static constexpr int TX_BYTES = E_BYTES + N_BYTES + K_BYTES + M_BYTES;  // + U_BYTES when u is staged
  static constexpr int O_BYTES = al(U_BYTES);   // one output staging buffer
  static int smem(int S) { return S * STAGE + 2 * O_BYTES + 8 * S + 128; }
};

template <typename T>
struct FusedArgs {
  using V = typename cplx<T>::t;
  const V* x;
  const double* omega;
  int* err;                  // the grid's error word: 1 = a bounded wait ran out, 2 = aborted
  const volatile int* abort; // the grid's abort word (pinned host memory), polled in every bounded wait
  const volatile int* abort_first;  // its device-memory copy, read once when the first copies are issued
  int nx, ny, nz, tz, nzc, ntx, nty, ntiles;
  int nb;    // systems in the batch; tile t = (chunk, row, column) * nb + b, so that CTAs running at the
             // same time work on one column for several systems and share its coefficients in L2
  int pf;    // L2 prefetch distance in planes ahead of the plane being loaded (0: none)
  int flat;  // 1: one system, the (column, plane) pairs split evenly over the CTAs (see ws kernel)
  long long ne;
  T out_scale;
};

// ---- masking of a staged e plane -------------------------------------------------------------------
// Edges on PEC walls and inside PEC cells are identity rows and zero columns of A, so their x values
// must not enter the curl: the staged e plane (cells i0-2 .. i0+TX+1, rows j0-1 .. j0+TY) is zeroed
// where the mask says so.  The staged mask row covers cells i0-16 .. i0+TX+15, so the e columns
// are mask bytes 14 .. TX+17, i.e. 32-bit words 3 .. 12 of each row (the outer halves of words 3
// and 12 belong to cells outside the e row).  NT threads share the plane; every thread loads its
// words first (independent loads, no per-row vote), and only a nonzero word costs any stores.
template <typename L, int NT>
__device__ inline void zero_masked_plane(typename L::V* e, const uint8_t* m, int t) {
  using V = typename L::V;
  constexpr int NWR = 10, NWORDS = L::ER * NWR, ROUNDS = (NWORDS + NT - 1) / NT;
  static_assert(TX == 32 && L::MW % 4 == 0 && 4 * (3 + NWR) <= L::MW, "mask row layout: 36 staged columns");
  uint32_t wv[ROUNDS];
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int idx = t + NT * r;
    uint32_t v = 0u;
    if (idx < NWORDS) {
      const int cy = idx / NWR, wi = 3 + idx % NWR;
      v = reinterpret_cast<const uint32_t*>(m + cy * L::MW)[wi];
      if (wi == 3) v &= 0xFFFF0000u;
      if (wi == 3 + NWR - 1) v &= 0x0000FFFFu;
    }
    wv[r] = v;
  }
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    if (wv[r] == 0u) continue;
    const int idx = t + NT * r;
    const int cy = idx / NWR, wi = 3 + idx % NWR;
#pragma unroll
    for (int bi = 0; bi < 4; ++bi) {
      const uint32_t mb = (wv[r] >> (8 * bi)) & 0xFFu;
      if (mb) {
        V* ec = e + cy * L::EW + 3 * (4 * wi + bi - 14);
        if (mb & 1u) ec[0] = czero<V>();
        if (mb & 2u) ec[1] = czero<V>();
        if (mb & 4u) ec[2] = czero<V>();
      }
    }
  }
}

// ---- PTX helpers: mbarrier and bulk tensor copies -----------------------------------------------
__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ inline void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false after ~2^22 polls (the copy engine never needs that long for a few KB), or as
// soon as the host sets the abort word (read every 4096 polls; abort = nullptr: no early exit, for the
// waits that let a CTA's own copies land before it leaves)
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* abort) {
  for (int it = 0; it < (1 << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(64);
    if ((it & 4095) == 4095 && abort && *abort) return false;
  }
  return false;
}
// the error code a kernel records when a wait gives up: 2 if the host asked it to stop, else 1.  Codes
// are recorded with atomicMax, so an abort seen by any role of any CTA wins over the timeouts it causes
// in the others.
__device__ inline int wait_error(const volatile int* abort) { return *abort ? 2 : 1; }
__device__ inline void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ inline void tma_load_4d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_u32(dst)), "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
// bulk tensor prefetch into L2 (no shared memory, no barrier): a later load of the same box hits L2
__device__ inline void tma_prefetch_3d(const CUtensorMap* tm, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(tm), "r"(c0), "r"(c1),
               "r"(c2)
               : "memory");
}
__device__ inline void tma_prefetch_4d(const CUtensorMap* tm, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(tm), "r"(c0), "r"(c1),
               "r"(c2), "r"(c3)
               : "memory");
}
// bulk tensor store from shared memory (coordinates are never negative here)
__device__ inline void tma_store_4d(const CUtensorMap* tm, const void* src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
               ::"l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ inline void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

__device__ inline void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---- the kernel ----------------------------------------------------------------------------------
// Persistent: the grid holds one wave of CTAs; CTA c processes tiles c, c + gridDim.x, ...
// (tile = x-tile, y-tile, z-chunk, system; x fastest).  The plane counter G and the output counter
// O run across tiles, so ring-stage parities and output buffers stay consistent.
template <typename T, int TY, int EPI, int S>
__global__ void __launch_bounds__(TX* TY, TY == 4 ? 5 : (TY == 8 ? 3 : 1)) fused_apply_kernel(const __grid_constant__ CUtensorMap tm_x,
                                                                const __grid_constant__ CUtensorMap tm_y,
                                                                const __grid_constant__ CUtensorMap tm_u,
                                                                const __grid_constant__ CUtensorMap tm_nu,
                                                                const __grid_constant__ CUtensorMap tm_ek,
                                                                const __grid_constant__ CUtensorMap tm_mask,
                                                                FusedArgs<T> a, fit_epi epi) {
  using V = typename cplx<T>::t;
  constexpr bool kU = (EPI == FIT_EPI_DOT_U || EPI == FIT_EPI_RESID);
  using L = Layout<T, TY, kU>;
  constexpr uint32_t kTx = L::TX_BYTES + (kU ? L::U_BYTES : 0);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  V* obuf = (V*)(smem + S * L::STAGE);  // two output staging buffers of O_BYTES
  uint64_t* bars = (uint64_t*)(smem + S * L::STAGE + 2 * L::O_BYTES);
  __shared__ int bad;

  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
    bad = 0;
  }
  __syncthreads();
  bool first_tile = true;

  unsigned G = 0, O = 0;        // planes issued into the ring / output planes written, this CTA
  bool pend = false;            // an output plane is staged but not yet stored (thread 0's view)
  int pi0 = 0, pj0 = 0, pk = 0, pb = 0;
  auto stage = [&](unsigned gq) -> unsigned char* { return smem + (gq % S) * L::STAGE; };
  const int er = (ty + 1) * L::EW + 3 * (tx + 2);
  const int nr = (ty + 1) * L::NW + 3 * (tx + 4);

  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int b = t % a.nb, c = t / a.nb;
    const int bx = c % a.ntx, by = (c / a.ntx) % a.nty, zc = c / (a.ntx * a.nty);
    if (epi.status && epi.status[b] != 0) continue;  // uniform over the CTA
    const int i0 = bx * TX, j0 = by * TY;
    const int k0 = zc * a.tz, k1 = min(a.nz, k0 + a.tz);
    const int nplanes = k1 - k0 + 2;  // planes k0-1 .. k1
    const unsigned G0 = G;

    auto issue = [&](int q) {  // thread 0 only
      const int p = k0 - 1 + q;
      unsigned char* st = stage(G0 + q);
      uint64_t* bar = &bars[(G0 + q) % S];
      mbar_expect_tx(bar, kTx);
      tma_load_4d(st + L::E_OFF, &tm_x, L::CE * 3 * (i0 - 2), j0 - 1, p, b, bar);
      tma_load_3d(st + L::N_OFF, &tm_nu, 3 * (i0 - 4), j0 - 1, p, bar);
      tma_load_3d(st + L::K_OFF, &tm_ek, 6 * i0, j0, p, bar);
      tma_load_3d(st + L::M_OFF, &tm_mask, i0 - 16, j0 - 1, p, bar);
      if (kU) tma_load_4d(st + L::U_OFF, &tm_u, L::CE * 3 * i0, j0, p, b, bar);
    };
    auto prefetch = [&](int q) {  // thread 0 only: the boxes of plane q into L2
      if (q >= nplanes) return;
      const int p = k0 - 1 + q;
      tma_prefetch_4d(&tm_x, L::CE * 3 * (i0 - 2), j0 - 1, p, b);
      tma_prefetch_3d(&tm_nu, 3 * (i0 - 4), j0 - 1, p);
      tma_prefetch_3d(&tm_ek, 6 * i0, j0, p);
      tma_prefetch_3d(&tm_mask, i0 - 16, j0 - 1, p);
      if (kU) tma_prefetch_4d(&tm_u, L::CE * 3 * i0, j0, p, b);
    };
    auto wait = [&](int q) {
      if (!mbar_wait(&bars[(G0 + q) % S], ((G0 + q) / S) & 1, a.abort)) {
        atomicMax(a.err, wait_error(a.abort));
        bad = 1;
      }
    };
    auto zero_pass = [&](int q) {  // P: zero masked components of the staged e plane
      zero_masked_plane<L, TX * TY>((V*)(stage(G0 + q) + L::E_OFF), stage(G0 + q) + L::M_OFF, tid);
      fence_proxy_async();  // order these generic writes before later bulk copies into the stage
    };

    if (tid == 0) {
      for (int q = 0; q < min(S, nplanes); ++q) issue(q);
      for (int q = S; q < S + a.pf; ++q) prefetch(q);  // the planes after the first ring fill
      // The abort word's device-memory copy is read once, after the first copies are on their way, so
      // that its latency hides under theirs; the barrier below publishes the answer before anything
      // is written.
      if (first_tile && *a.abort_first) {
        bad = 1;
        atomicMax(a.err, 2);
      }
    }
    first_tile = false;
    int issued = min(S, nplanes);
    auto drain = [&]() {  // bounded waits for every copy this tile issued
      for (int q = 0; q < issued; ++q) (void)mbar_wait(&bars[(G0 + q) % S], ((G0 + q) / S) & 1, nullptr);
    };

    // prologue: planes k0-1 (q = 0) and k0 (q = 1); h(k0-1) of the own column
    wait(0);
    zero_pass(0);
    wait(1);
    zero_pass(1);
    __syncthreads();
    if (bad) {
      drain();
      break;
    }
    V e0[3], em[3], ejm[3];
    V hxp, hyp;
    {
      const V* p0 = (const V*)(stage(G0) + L::E_OFF) + er;
      const V* p1 = (const V*)(stage(G0 + 1) + L::E_OFF) + er;
      const T* n0 = (const T*)(stage(G0) + L::N_OFF) + nr;
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        e0[w] = p1[w];
        em[w] = p1[w - 3];
        ejm[w] = p1[w - L::EW];
      }
      hxp = n0[0] * (p0[1] - e0[1] + p0[L::EW + 2] - p0[2]);
      hyp = n0[1] * (p0[2] - p0[3 + 2] + e0[0] - p0[0]);
    }

    T acc[3] = {T(0), T(0), T(0)};
    const double wd = a.omega[b];
    const T w1 = (T)wd, w2 = (T)(wd * wd);
    const V* xg = a.x + (long long)b * a.ne;
    const int i = i0 + tx, j = j0 + ty;
    const bool valid = i < a.nx && j < a.ny;

    for (int k = k0; k < k1; ++k) {
      const int qk = k - k0 + 1, qn = qk + 1;
      wait(qn);
      zero_pass(qn);
      if (tid == 0) bulk_wait_read_all();  // the output buffer written this step is free again
      __syncthreads();
      if (bad) break;
      if (tid == 0) {
        if (pend) tma_store_4d(&tm_y, obuf + (size_t)((O - 1) & 1) * (L::O_BYTES / sizeof(V)),
                               L::CE * 3 * pi0, pj0, pk, pb);
        if (qk - 1 + S < nplanes) {
          issue(qk - 1 + S);  // plane qk-1 is released by the barrier above
          if (a.pf) prefetch(qk - 1 + S + a.pf);
        }
      }
      pend = false;
      if (qk - 1 + S < nplanes) issued = qk + S;
      // ---- this thread's column at plane k ----
      const unsigned char* s0 = stage(G0 + qk);
      const V* p0 = (const V*)(s0 + L::E_OFF) + er;
      const V* p1 = (const V*)(stage(G0 + qn) + L::E_OFF) + er;
      const T* nn = (const T*)(s0 + L::N_OFF) + nr;
      V e1[3], em1[3], ejm1[3];
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        e1[w] = p1[w];
        em1[w] = p1[w - 3];
        ejm1[w] = p1[w - L::EW];
      }
      const V ez_jp = p0[L::EW + 2], ex_jp = p0[L::EW];
      const V ez_ip = p0[3 + 2], ey_ip = p0[3 + 1];
      const V ex_imjp = p0[L::EW - 3], ey_ipjm = p0[3 + 1 - L::EW];
      const V hx = nn[0] * (e0[1] - e1[1] + ez_jp - e0[2]);
      const V hy = nn[1] * (e0[2] - ez_ip + e1[0] - e0[0]);
      const V hz = nn[2] * (e0[0] - ex_jp + ey_ip - e0[1]);
      const V hy_im = nn[1 - 3] * (em[2] - e0[2] + em1[0] - em[0]);
      const V hz_im = nn[2 - 3] * (em[0] - ex_imjp + e0[1] - em[1]);
      const V hx_jm = nn[0 - L::NW] * (ejm[1] - ejm1[1] + e0[2] - ejm[2]);
      const V hz_jm = nn[2 - L::NW] * (ejm[0] - e0[0] + ey_ipjm - ejm[1]);
      V curl[3];
      curl[0] = hyp - hy + hz - hz_jm;
      curl[1] = hz_im - hz + hx - hxp;
      curl[2] = hx_jm - hx + hy - hy_im;
      const T* ek = (const T*)(s0 + L::K_OFF) + ty * L::KW + 6 * tx;
      const uint8_t m = (s0 + L::M_OFF)[(ty + 1) * L::MW + tx + 16];
      const V* uv = (const V*)(s0 + L::U_OFF) + ty * L::OW + 3 * tx;
      V* ob = obuf + (size_t)(O & 1) * (L::O_BYTES / sizeof(V)) + ty * L::OW + 3 * tx;
      const long long cbase = 3 * (i + (long long)a.nx * (j + (long long)a.ny * k));
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        V out;
        V xv = e0[w];
        if ((m >> w) & 1) {
          xv = valid ? xg[cbase + w] : czero<V>();  // raw x on a masked edge
          out = xv;
        } else {
          const T ar = -w2 * ek[w], ai = w1 * ek[3 + w];
          out.x = a.out_scale * (curl[w].x + ar * xv.x - ai * xv.y);
          out.y = a.out_scale * (curl[w].y + ar * xv.y + ai * xv.x);
        }
        if (EPI == FIT_EPI_RESID) out = uv[w] - out;
        if (valid) {
          if (EPI == FIT_EPI_DOT_U) {
            acc[0] += uv[w].x * out.x + uv[w].y * out.y;
            acc[1] += uv[w].x * out.y - uv[w].y * out.x;
          } else if (EPI == FIT_EPI_DOT_TS) {
            acc[0] += out.x * xv.x + out.y * xv.y;
            acc[1] += out.x * xv.y - out.y * xv.x;
            acc[2] += out.x * out.x + out.y * out.y;
          } else if (EPI == FIT_EPI_RESID) {
            acc[2] += out.x * out.x + out.y * out.y;
          } else if (EPI == FIT_EPI_DOT_XY) {
            acc[0] += xv.x * out.x - xv.y * out.y;
            acc[1] += xv.x * out.y + xv.y * out.x;
          }
        }
        ob[w] = out;
      }
      fence_proxy_async();  // the bulk store issued after the next barrier reads these values
      pend = true;
      pi0 = i0;
      pj0 = j0;
      pk = k;
      pb = b;
      ++O;
      hxp = hx;
      hyp = hy;
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        e0[w] = e1[w];
        em[w] = em1[w];
        ejm[w] = ejm1[w];
      }
    }
    if (bad) {  // a copy did not complete in time: drain what this tile issued and stop
      drain();
      break;
    }
    G += nplanes;
    __syncthreads();  // stages free for the next tile; the last output plane is staged
    if (tid == 0 && pend) tma_store_4d(&tm_y, obuf + (size_t)((O - 1) & 1) * (L::O_BYTES / sizeof(V)),
                                       L::CE * 3 * pi0, pj0, pk, pb);
    pend = false;
    if (EPI != FIT_EPI_NONE) {
      const long long nblk = (long long)a.ntx * a.nty * a.nzc;
      const long long blk = ((long long)zc * a.nty + by) * a.ntx + bx;
      fit_block_sum<T, 3>(acc, epi.part + ((long long)b * nblk + blk) * 4);
    }
  }
  if (tid == 0) bulk_wait_all();  // every output store has landed before the CTA retires
}


// ---- warp-specialised variant -------------------------------------------------------------------
// Warps 0..TY-1 are consumers (one tile row each), warp TY issues the bulk copies (lane 0) and warp
// TY+1 masks the staged planes.  Per ring stage s:
//   full[s]  (1 arrival + bytes): the bulk copies of a plane have landed
//   ready[s] (1 arrival): the masking warp has zeroed the plane's masked edges; consumers may read it
//   empty[s] (TY arrivals): every consumer warp is done with the plane; the stage may be refilled
// The issuing warp waits on nothing but empty[], so a stage is refilled as soon as it is released
// (consumers release plane k right after their shared-memory reads of it, before the arithmetic);
// the masking warp waits on nothing but full[].  Plane p needs the release of plane p - S, which
// the consumers give after their step p - S (planes p - S and p - S + 1), so no role waits on work
// that depends on its own later progress.  No CTA-wide barrier is needed in the steady state, and
// the issuing warp runs into the next tile while the consumers finish the current one.
__device__ inline uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for a handoff between warps of the CTA: spin on try_wait (which itself suspends the thread
// until the phase completes or a short hardware limit passes) with no sleep in between, so the
// waiting warp resumes as soon as the other side arrives; gives up 0.5 s of wall time after its 256th
// poll.  The clock is first read at that poll, not on entry, so a handoff that completes sooner (every
// handoff of a healthy apply) never waits on a timer read.  The host's abort word ends a wait that has
// already lasted 20 us more (far beyond any handoff of a running apply, so the word, in host memory,
// is never read on the way of a healthy kernel); abort = nullptr for the waits that let the CTA's own
// copies land before it leaves.
__device__ inline bool mbar_wait_handoff(uint64_t* bar, uint32_t parity, const volatile int* abort) {
  uint64_t t0 = 0;
  for (uint32_t it = 1; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0u) {
      const uint64_t now = global_ns();
      if (it == 256u) {
        t0 = now;
        continue;
      }
      const uint64_t dt = now - t0;
      if (dt > 500000000ull || (abort && dt > 20000ull && *abort)) return false;
    }
  }
  return false;
}
__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ inline void named_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// resident CTAs per SM the register budget is sized for: about 20 warps per SM for complex64
template <typename T, int TY>
constexpr int ws_min_blocks() {
  return sizeof(T) == 4 ? (20 / (TY + 2) > 1 ? 20 / (TY + 2) : 1) : 1;
}

template <typename T, int TY, int EPI, int S>
__global__ void __launch_bounds__(TX*(TY + 2), ws_min_blocks<T, TY>()) ws_apply_kernel(const __grid_constant__ CUtensorMap tm_x,
                                                                  const __grid_constant__ CUtensorMap tm_u,
                                                                  const __grid_constant__ CUtensorMap tm_nu,
                                                                  const __grid_constant__ CUtensorMap tm_ek,
                                                                  const __grid_constant__ CUtensorMap tm_mask,
                                                                  FusedArgs<T> a, typename cplx<T>::t* yout, fit_epi epi) {
  using V = typename cplx<T>::t;
  constexpr bool kU = (EPI == FIT_EPI_DOT_U || EPI == FIT_EPI_RESID);
  using L = Layout<T, TY, kU>;
  constexpr uint32_t kTx = L::TX_BYTES + (kU ? L::U_BYTES : 0);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  V* stg_all = (V*)(smem + S * L::STAGE);                           // per consumer warp: 96 values
  uint64_t* full = (uint64_t*)(smem + S * L::STAGE + L::O_BYTES);   // O_BYTES >= TY*96*sizeof(V)
  uint64_t* ready = full + S;
  uint64_t* empty = ready + S;
  uint64_t* checked = empty + S;                                     // the abort word has been read
  double* red = (double*)(checked + 1);                              // [TY][3] tile partial sums
  volatile int* abort_flag = (volatile int*)(red + 3 * TY);
  volatile int* quit = abort_flag + 1;                               // the abort word was set at start

  const int lane = threadIdx.x, warp = threadIdx.y;
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], 1);
      mbar_init(&empty[s], TY);
    }
    mbar_init(checked, 1);
    *abort_flag = 0;
    *quit = 0;
    fence_mbar_init();
  }
  __syncthreads();
  auto stage = [&](unsigned gq) -> unsigned char* { return smem + (gq % S) * L::STAGE; };
  // the issuing and masking warps read the abort word when they give up; a consumer warp only gives up
  // after them (its planes stop arriving), so it records a plain timeout and leaves the abort code to
  // them (and keeps the host word's address out of its registers)
  auto fail = [&]() { atomicMax(a.err, wait_error(a.abort)); };
  auto fail_consumer = [&]() { atomicMax(a.err, 1); };

  // This CTA's work, one segment (bx, by, b, planes k0 .. k1-1) at a time; every role walks the
  // same sequence.  Tiled: tiles blockIdx.x, blockIdx.x + gridDim.x, ... of ntx*nty*nzc*nbatch
  // chunks of tz planes, the system index fastest; the partial sums of a tile go to its own slot.  Flat (one system): the
  // ntx*nty*nz (column, plane) pairs, column-major, are cut into gridDim.x equal contiguous ranges,
  // one per CTA, so every resident CTA gets the same work; a range may cover the end of one column
  // and the start of the next, and the CTA's partial sums go to slot blockIdx.x once at the end.
  // (ntx*nty*nz is below 2^31 for any grid that fits in device memory: 32 x TY cells per column)
  int wpos = 0, wend = 0;
  int tnext = blockIdx.x;
  if (a.flat) {
    const long long W = (long long)a.ntx * a.nty * a.nz;
    wpos = (int)(W * blockIdx.x / gridDim.x);
    wend = (int)(W * (blockIdx.x + 1) / gridDim.x);
  }
  auto next = [&](int& bx, int& by, int& b, int& k0, int& k1, int& slot) -> bool {
    if (a.flat) {
      if (wpos >= wend) return false;
      const int col = wpos / a.nz;
      k0 = wpos - col * a.nz;
      k1 = min(a.nz, k0 + (wend - wpos));
      wpos += k1 - k0;
      bx = col % a.ntx;
      by = col / a.ntx;
      b = 0;
      slot = blockIdx.x;
      return true;
    }
    if (tnext >= a.ntiles) return false;
    const int t = tnext;
    tnext += gridDim.x;
    b = t % a.nb;
    const int c = t / a.nb;
    bx = c % a.ntx;
    by = (c / a.ntx) % a.nty;
    const int zc = c / (a.ntx * a.nty);
    k0 = zc * a.tz;
    k1 = min(a.nz, k0 + a.tz);
    slot = (zc * a.nty + by) * a.ntx + bx;
    return true;
  };

  if (warp == TY) {
    // ---------------- issuing warp: lane 0 refills released stages ----------------
    if (lane != 0) return;
    unsigned G = 0;
    int bx, by, b, k0, k1, slot;
    bool checked_abort = false;
    // The abort word (its device-memory copy) is loaded before the first copies are issued and used
    // after them, so that its latency hides under theirs; the masking warp waits for the answer before
    // it releases any plane to the consumers, so a kernel that starts aborted writes nothing.
    const int abort_at_start = *a.abort_first;
    auto check_abort = [&]() -> bool {  // returns true if the CTA must stop
      checked_abort = true;
      const bool stop = abort_at_start != 0;
      if (stop) {
        *quit = 1;
        atomicMax(a.err, 2);
      }
      mbar_arrive(checked);
      return stop;
    };
    auto drain_all = [&]() {  // every copy this warp issued lands before the CTA retires
      for (unsigned d = 1; d <= S && d <= G; ++d) (void)mbar_wait_handoff(&full[(G - d) % S], ((G - d) / S) & 1, nullptr);
    };
    while (next(bx, by, b, k0, k1, slot)) {
      if (epi.status && epi.status[b] != 0) continue;  // the same skip in every role
      const int i0 = bx * TX, j0 = by * TY;
      auto prefetch = [&](int p) {  // the boxes of plane p into L2
        if (p > k1) return;
        tma_prefetch_4d(&tm_x, L::CE * 3 * (i0 - 2), j0 - 1, p, b);
        tma_prefetch_3d(&tm_nu, 3 * (i0 - 4), j0 - 1, p);
        tma_prefetch_3d(&tm_ek, 6 * i0, j0, p);
        tma_prefetch_3d(&tm_mask, i0 - 16, j0 - 1, p);
        if (kU) tma_prefetch_4d(&tm_u, L::CE * 3 * i0, j0, p, b);
      };
      // the tile's first planes wait for stages the previous tile still holds: start them in L2
      if (a.pf)
        for (int p = k0 - 1; p < k0 - 1 + S + a.pf; ++p) prefetch(p);
      for (int p = k0 - 1; p <= k1; ++p, ++G) {
        const unsigned s = G % S, use = G / S;
        if (use > 0 && !checked_abort && check_abort()) {
          drain_all();
          return;
        }
        if (use > 0 && !mbar_wait_handoff(&empty[s], (use - 1) & 1, a.abort)) {
          // record; the copies still in flight are the last (at most S - 1) issued: let them land
          fail();
          for (unsigned d = 1; d <= S && d <= G; ++d) (void)mbar_wait_handoff(&full[(G - d) % S], ((G - d) / S) & 1, nullptr);
          return;
        }
        unsigned char* st = stage(G);
        mbar_expect_tx(&full[s], kTx);
        tma_load_4d(st + L::E_OFF, &tm_x, L::CE * 3 * (i0 - 2), j0 - 1, p, b, &full[s]);
        tma_load_3d(st + L::N_OFF, &tm_nu, 3 * (i0 - 4), j0 - 1, p, &full[s]);
        tma_load_3d(st + L::K_OFF, &tm_ek, 6 * i0, j0, p, &full[s]);
        tma_load_3d(st + L::M_OFF, &tm_mask, i0 - 16, j0 - 1, p, &full[s]);
        if (kU) tma_load_4d(st + L::U_OFF, &tm_u, L::CE * 3 * i0, j0, p, b, &full[s]);
        if (a.pf && p - (k0 - 1) >= S) prefetch(p + a.pf);
      }
      if (!checked_abort && check_abort()) {  // a first segment shorter than the ring
        drain_all();
        return;
      }
    }
    if (!checked_abort) mbar_arrive(checked);  // no work: nobody waits, but keep the protocol whole
    drain_all();
    return;
  }

  if (warp == TY + 1) {
    // ---------------- masking warp: zero the masked edges of each landed plane ----------------
    unsigned G = 0;
    int bx, by, b, k0, k1, slot;
    bool released = false;
    while (next(bx, by, b, k0, k1, slot)) {
      if (epi.status && epi.status[b] != 0) continue;
      const int nplanes = k1 - k0 + 2;
      if (!released) {  // nothing reaches the consumers before the issuing warp has read the abort word
        if (!__all_sync(0xffffffffu, mbar_wait_handoff(checked, 0, a.abort)) || *quit) {
          if (lane == 0) fail();
          return;
        }
        released = true;
      }
      for (int q = 0; q < nplanes; ++q, ++G) {
        if (!__all_sync(0xffffffffu, mbar_wait_handoff(&full[G % S], (G / S) & 1, a.abort))) {  // warp-uniform
          if (lane == 0) fail();
          return;
        }
        zero_masked_plane<L, 32>((V*)(stage(G) + L::E_OFF), stage(G) + L::M_OFF, lane);
        fence_proxy_async();  // these generic writes precede the stage's next bulk copy
        __syncwarp();
        if (lane == 0) mbar_arrive(&ready[G % S]);
      }
    }
    return;
  }

  // ---------------- consumer warps: row ty = warp ----------------
  // A warp whose wait timed out stops computing but still takes part in the partial-sum barriers,
  // so the other consumer warps never wait on it; all consumers leave together after the flush.
  T acc[3] = {T(0), T(0), T(0)};
  bool dead = false;
  // Reduce acc over the CTA's consumer rows (warp shuffles, then FP64 over the rows in order) into
  // part[(b * nslots + slot) * 4 + q]; returns true when the consumers must stop.
  auto flush = [&](int b, int slot, long long nslots) -> bool {
    if (dead) {
      fail_consumer();
      *abort_flag = 1;
    }
    if (EPI == FIT_EPI_NONE) return dead;  // no barrier: a dead warp leaves on its own
#pragma unroll
    for (int qq = 0; qq < 3; ++qq) {
      T v = acc[qq];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp * 3 + qq] = (double)v;
    }
    named_barrier(1, TX * TY);
    if (warp == 0 && lane < 3) {
      double sum = 0.0;
      for (int r = 0; r < TY; ++r) sum += red[r * 3 + lane];
      epi.part[((long long)b * nslots + slot) * 4 + lane] = sum;
    }
    named_barrier(1, TX * TY);
    return *abort_flag != 0;  // read after the barrier: the same answer in every consumer warp
  };
  unsigned G = 0;
  int bx, by, b, k0, k1, slot;
  while (next(bx, by, b, k0, k1, slot)) {
    if (epi.status && epi.status[b] != 0) continue;
    const int i0 = bx * TX, j0 = by * TY;
    const int nplanes = k1 - k0 + 2;  // planes k0-1 .. k1
    const unsigned G0 = G;
    {
      const int tx = lane, ty = warp;
      const int er = (ty + 1) * L::EW + 3 * (tx + 2);
      const int nr = (ty + 1) * L::NW + 3 * (tx + 4);
      V* stg = stg_all + ty * 96;
      dead = !mbar_wait_handoff(&ready[G0 % S], (G0 / S) & 1, nullptr) ||
             !mbar_wait_handoff(&ready[(G0 + 1) % S], ((G0 + 1) / S) & 1, nullptr);
      dead = __any_sync(0xffffffffu, dead);  // warp-uniform
      if (!dead) {
        V e0[3], em[3], ejm[3];
        V hxp, hyp;
        {
          const V* p0 = (const V*)(stage(G0) + L::E_OFF) + er;
          const V* p1 = (const V*)(stage(G0 + 1) + L::E_OFF) + er;
          const T* n0 = (const T*)(stage(G0) + L::N_OFF) + nr;
#pragma unroll
          for (int w = 0; w < 3; ++w) {
            e0[w] = p1[w];
            em[w] = p1[w - 3];
            ejm[w] = p1[w - L::EW];
          }
          hxp = n0[0] * (p0[1] - e0[1] + p0[L::EW + 2] - p0[2]);
          hyp = n0[1] * (p0[2] - p0[3 + 2] + e0[0] - p0[0]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[G0 % S]);  // plane k0-1 is no longer needed
        const double wd = a.omega[b];
        const T w1 = (T)wd, w2 = (T)(wd * wd);
        const long long boff = (long long)b * a.ne;
        const V* xg = a.x + boff;
        V* yg = yout + boff;
        const int i = i0 + tx, j = j0 + ty;
        const bool valid = i < a.nx && j < a.ny;
        const int nvalid = 3 * max(0, min(TX, a.nx - i0));
        // two planes per trip: the values carried from plane k to k+1 stay in place instead of being
        // copied between registers every step
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
          const int qk = k - k0 + 1, qn = qk + 1;
          // (the consumers' waits do not read the abort word: the issuing and masking warps do, and a
          // consumer whose planes stop arriving gives up on its own bound)
          if (__any_sync(0xffffffffu, !mbar_wait_handoff(&ready[(G0 + qn) % S], ((G0 + qn) / S) & 1, nullptr))) {
            dead = true;
            break;
          }
          const unsigned char* s0 = stage(G0 + qk);
          const V* p0 = (const V*)(s0 + L::E_OFF) + er;
          const V* p1 = (const V*)(stage(G0 + qn) + L::E_OFF) + er;
          const T* nn = (const T*)(s0 + L::N_OFF) + nr;
          V e1[3], em1[3], ejm1[3];
#pragma unroll
          for (int w = 0; w < 3; ++w) {
            e1[w] = p1[w];
            em1[w] = p1[w - 3];
            ejm1[w] = p1[w - L::EW];
          }
          // every value of plane qk this step needs, read before the plane is released
          const V ez_jp = p0[L::EW + 2], ex_jp = p0[L::EW];
          const V ez_ip = p0[3 + 2], ey_ip = p0[3 + 1];
          const V ex_imjp = p0[L::EW - 3], ey_ipjm = p0[3 + 1 - L::EW];
          const T nu_x = nn[0], nu_y = nn[1], nu_z = nn[2], nu_y_im = nn[1 - 3], nu_z_im = nn[2 - 3];
          const T nu_x_jm = nn[0 - L::NW], nu_z_jm = nn[2 - L::NW];
          T ek[6];
          const T* ekp = (const T*)(s0 + L::K_OFF) + ty * L::KW + 6 * tx;
#pragma unroll
          for (int c = 0; c < 6; ++c) ek[c] = ekp[c];
          const uint8_t m = (s0 + L::M_OFF)[(ty + 1) * L::MW + tx + 16];
          // without a staged u the plane is released before the arithmetic; with one, the u values
          // are read where they are used and the plane is released after the step (fewer live registers)
          const V* uv = (const V*)(s0 + L::U_OFF) + ty * L::OW + 3 * tx;
          if (!kU) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[(G0 + qk) % S]);  // plane qk is no longer needed
          }
          const V hx = nu_x * (e0[1] - e1[1] + ez_jp - e0[2]);
          const V hy = nu_y * (e0[2] - ez_ip + e1[0] - e0[0]);
          const V hz = nu_z * (e0[0] - ex_jp + ey_ip - e0[1]);
          const V hy_im = nu_y_im * (em[2] - e0[2] + em1[0] - em[0]);
          const V hz_im = nu_z_im * (em[0] - ex_imjp + e0[1] - em[1]);
          const V hx_jm = nu_x_jm * (ejm[1] - ejm1[1] + e0[2] - ejm[2]);
          const V hz_jm = nu_z_jm * (ejm[0] - e0[0] + ey_ipjm - ejm[1]);
          V curl[3];
          curl[0] = hyp - hy + hz - hz_jm;
          curl[1] = hz_im - hz + hx - hxp;
          curl[2] = hx_jm - hx + hy - hy_im;
          const long long rowbase = 3 * (i0 + (long long)a.nx * (j + (long long)a.ny * k));
#pragma unroll
          for (int w = 0; w < 3; ++w) {
            V out;
            V xv = e0[w];
            if ((m >> w) & 1) {
              xv = valid ? xg[rowbase + 3 * tx + w] : czero<V>();  // raw x on a masked edge
              out = xv;
            } else {
              const T ar = -w2 * ek[w], ai = w1 * ek[3 + w];
              out.x = a.out_scale * (curl[w].x + ar * xv.x - ai * xv.y);
              out.y = a.out_scale * (curl[w].y + ar * xv.y + ai * xv.x);
            }
            if (EPI == FIT_EPI_RESID) out = uv[w] - out;
            if (valid) {
              if (EPI == FIT_EPI_DOT_U) {
                acc[0] += uv[w].x * out.x + uv[w].y * out.y;
                acc[1] += uv[w].x * out.y - uv[w].y * out.x;
              } else if (EPI == FIT_EPI_DOT_TS) {
                acc[0] += out.x * xv.x + out.y * xv.y;
                acc[1] += out.x * xv.y - out.y * xv.x;
                acc[2] += out.x * out.x + out.y * out.y;
              } else if (EPI == FIT_EPI_RESID) {
                acc[2] += out.x * out.x + out.y * out.y;
              } else if (EPI == FIT_EPI_DOT_XY) {
                acc[0] += xv.x * out.x - xv.y * out.y;
                acc[1] += xv.x * out.y + xv.y * out.x;
              }
            }
            stg[3 * tx + w] = out;
          }
          __syncwarp();  // the staged output row is complete (and, with u, plane qk is read)
          if (kU && lane == 0) mbar_arrive(&empty[(G0 + qk) % S]);
          if (j < a.ny) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              const int q = tx + 32 * r;
              if (q < nvalid) yg[rowbase + q] = stg[q];
            }
          }
          __syncwarp();
          hxp = hx;
          hyp = hy;
#pragma unroll
          for (int w = 0; w < 3; ++w) {
            e0[w] = e1[w];
            em[w] = em1[w];
            ejm[w] = ejm1[w];
          }
        }
        if (!dead && lane == 0) mbar_arrive(&empty[(G0 + nplanes - 1) % S]);  // plane k1 (read as k+1 only)
      }
    }
    G += nplanes;
    if (!a.flat) {  // the tile's own slot
      if (flush(b, slot, (long long)a.ntx * a.nty * a.nzc)) return;
      acc[0] = acc[1] = acc[2] = T(0);
    } else if (dead) {
      break;
    }
  }
  if (a.flat) (void)flush(0, blockIdx.x, gridDim.x);
}

// ---- host side -----------------------------------------------------------------------------------
typedef CUresult (*encode_fn_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_fn_t encoder() {
  static encode_fn_t fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (encode_fn_t)p;
  }
  return fn;
}

bool encode(CUtensorMap* m, CUtensorMapDataType dt, int rank, const void* base, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box) {
  encode_fn_t fn = encoder();
  if (!fn) return false;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = fn(m, dt, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

struct Variant {
  int ty, tz, stages, ws, pf;  // ws: warp-specialised kernel; pf: L2 prefetch distance (planes)
};
// candidate launch shapes; the autotuner picks one per (grid, precision, batch)
// tz = 0: chunk length chosen at launch so that the tiles fill the resident CTAs in one balanced wave
// tz = -1 (warp-specialised kernel, one system): the (column, plane) pairs split evenly over the
//         resident CTAs; with a batch it falls back to tz = 0
const Variant kVariants64[] = {
    {8, 16, 4, 0, 0}, {4, 32, 4, 0, 0}, {4, 0, 3, 0, 0}, {4, 0, 4, 0, 0}, {8, 0, 3, 0, 0}, {8, 0, 4, 0, 0},
    {8, 0, 3, 0, 2},  {8, 0, 3, 0, 4},  {8, 0, 3, 0, 8}, {4, 0, 4, 0, 4}, {8, 0, 4, 0, 4},
    {4, 0, 4, 1, 0},  {8, 0, 4, 1, 0},  {8, 32, 4, 1, 0}, {16, 0, 4, 1, 0},
    {4, 0, 4, 1, 4},  {8, 0, 3, 1, 4},  {8, 0, 4, 1, 2}, {8, 0, 4, 1, 4}, {8, 0, 4, 1, 8}, {8, 32, 4, 1, 4},
    {8, -1, 4, 1, 0}, {4, -1, 4, 1, 0}, {8, -1, 4, 1, 2},
    // taller tiles and deeper rings on the even split: fewer y-halo rows per cell, longer z ranges per CTA
    {16, -1, 4, 1, 0}, {16, -1, 5, 1, 0}, {16, -1, 4, 1, 2}, {8, -1, 5, 1, 0}, {8, -1, 3, 1, 0}};
const Variant kVariants128[] = {{4, 16, 3, 0, 0}, {4, 32, 3, 0, 0}, {8, 16, 3, 0, 0}, {8, 32, 3, 0, 0},
                                {4, 0, 3, 0, 0},  {8, 0, 3, 0, 0},  {4, 0, 4, 1, 0},  {8, 0, 4, 1, 0},
                                {8, 0, 3, 0, 4},  {4, 0, 4, 1, 4},  {8, 0, 4, 1, 4},  {8, -1, 4, 1, 0}};

// largest dynamic shared memory a CTA may opt in to on the current device
int fused_smem_limit() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 0;
  return v;
}

// dynamic shared memory of a variant with the largest epilogue staging (the vector u of DOT_U / RESID)
template <typename T, int TY, int S, int WS>
int variant_smem_max() {
  return Layout<T, TY, true>::smem(S) + (WS ? 3 * 8 * S + 8 * 3 * TY + 16 : 0);
}

template <typename T, int TY, int S, int WS>
fit_status launch_variant(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y, const T* nu,
                          const T* ek, double out_scale, cudaStream_t s, fit_epi& e, int tz, int pf) {
  const bool c64 = sizeof(T) == 4;
  CUtensorMap mx, mnu, mek, mmask;
  const cuuint64_t ce = c64 ? 1 : 2;
  {
    cuuint64_t dims[4] = {3 * ce * (cuuint64_t)g->nx, (cuuint64_t)g->ny, (cuuint64_t)g->nz, (cuuint64_t)nbatch};
    cuuint64_t rowb = 3 * ce * 8 * (cuuint64_t)g->nx;
    cuuint64_t str[3] = {rowb, rowb * g->ny, rowb * g->ny * g->nz};
    cuuint32_t box[4] = {(cuuint32_t)(3 * ce * (TX + 4)), TY + 2, 1, 1};
    if (!encode(&mx, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, x, dims, str, box)) {
      fit_set_error("fused apply: tensor map of x rejected");
      return FIT_ECUDA;
    }
  }
  const CUtensorMapDataType cdt = c64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  {
    cuuint64_t dims[3] = {3 * (cuuint64_t)g->nxp, (cuuint64_t)g->ny, (cuuint64_t)g->nz};
    cuuint64_t rowb = 3 * sizeof(T) * (cuuint64_t)g->nxp;
    cuuint64_t str[2] = {rowb, rowb * g->ny};
    cuuint32_t box[3] = {3 * (TX + 4), TY + 1, 1};
    if (!encode(&mnu, cdt, 3, nu, dims, str, box)) {
      fit_set_error("fused apply: tensor map of M_nu rejected");
      return FIT_ECUDA;
    }
  }
  {
    cuuint64_t dims[3] = {6 * (cuuint64_t)g->nxp, (cuuint64_t)g->ny, (cuuint64_t)g->nz};
    cuuint64_t rowb = 6 * sizeof(T) * (cuuint64_t)g->nxp;
    cuuint64_t str[2] = {rowb, rowb * g->ny};
    cuuint32_t box[3] = {6 * TX, TY, 1};
    if (!encode(&mek, cdt, 3, ek, dims, str, box)) {
      fit_set_error("fused apply: tensor map of M_eps/M_kappa rejected");
      return FIT_ECUDA;
    }
  }
  {
    cuuint64_t dims[3] = {(cuuint64_t)g->nxp, (cuuint64_t)g->ny, (cuuint64_t)g->nz};
    cuuint64_t str[2] = {(cuuint64_t)g->nxp, (cuuint64_t)g->nxp * g->ny};
    cuuint32_t box[3] = {TX + 32, TY + 2, 1};
    if (!encode(&mmask, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, g->mask, dims, str, box)) {
      fit_set_error("fused apply: tensor map of the mask rejected");
      return FIT_ECUDA;
    }
  }
  // y (bulk tensor store, box of the own cells) and the epilogue vector u (same shape as x)
  CUtensorMap my, mu;
  {
    cuuint64_t dims[4] = {3 * ce * (cuuint64_t)g->nx, (cuuint64_t)g->ny, (cuuint64_t)g->nz, (cuuint64_t)nbatch};
    cuuint64_t rowb = 3 * ce * 8 * (cuuint64_t)g->nx;
    cuuint64_t str[3] = {rowb, rowb * g->ny, rowb * g->ny * g->nz};
    cuuint32_t box[4] = {(cuuint32_t)(3 * ce * TX), TY, 1, 1};
    if (!encode(&my, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, y, dims, str, box)) {
      fit_set_error("fused apply: tensor map of y rejected");
      return FIT_ECUDA;
    }
    const void* ub = (e.mode == FIT_EPI_DOT_U || e.mode == FIT_EPI_RESID) ? e.u : x;
    if (((uintptr_t)ub & 15) != 0 || !encode(&mu, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, ub, dims, str, box)) {
      fit_set_error("fused apply: tensor map of the epilogue vector rejected");
      return FIT_ECUDA;
    }
  }
  FusedArgs<T> a;
  a.x = (const typename cplx<T>::t*)x;
  a.omega = omega_dev;
  a.err = g->err_dev;
  a.abort = g->abort_dev;
  a.abort_first = g->abort_mirror;
  a.nx = g->nx;
  a.ny = g->ny;
  a.nz = g->nz;
  a.ntx = (g->nx + TX - 1) / TX;
  a.nty = (g->ny + TY - 1) / TY;
  a.ne = g->ne;
  a.out_scale = (T)out_scale;
  a.pf = pf;
  a.flat = 0;
  a.nb = nbatch;
  dim3 block(TX, WS ? TY + 2 : TY, 1);
  const bool ku = e.mode == FIT_EPI_DOT_U || e.mode == FIT_EPI_RESID;
  int smem = ku ? Layout<T, TY, true>::smem(S) : Layout<T, TY, false>::smem(S);
  if (WS) smem += 3 * 8 * S + 8 + 8 * 3 * TY + 16;  // three barriers per stage, the abort check, row sums, flags
  auto run = [&](auto kern) -> fit_status {
    if (smem > fused_smem_limit()) {  // this ring depth and epilogue staging exceed an SM's shared memory
      fit_set_error("fused apply: launch shape does not fit on an SM");
      return FIT_EINVAL;
    }
    FIT_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0, nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    FIT_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block.x * block.y, smem));
    if (per_sm < 1) {  // shared memory or registers do not allow one resident CTA of this shape
      fit_set_error("fused apply: launch shape does not fit on an SM");
      return FIT_EINVAL;
    }
    const long long slots = (long long)per_sm * nsm;
    int grid = 0;
    a.flat = 0;
    if (WS && tz < 0 && nbatch == 1) {
      // one system: every resident CTA takes an equal share of the (column, plane) pairs; at most
      // ntx*nty*ceil(nz/2) CTAs (ranges of about two planes or more, and within the partial-sum
      // buffer, which is sized for chunks of two planes)
      const long long cap = (long long)a.ntx * a.nty * ((g->nz + 1) / 2);
      grid = (int)std::max(1LL, std::min(slots, cap));
      a.flat = 1;
      a.tz = 0;
      a.nzc = 0;
      a.ntiles = 0;
      e.nslots = grid;
    } else {
      int tzz = tz;
      if (tzz <= 0) {  // balanced: as many equal z-chunks per column tile as the resident CTAs allow
        const long long cols = (long long)a.ntx * a.nty * nbatch;
        const long long per_col = std::max(1LL, slots / std::max(1LL, cols));
        tzz = (int)std::max(2LL, ((long long)g->nz + per_col - 1) / per_col);
      }
      a.tz = tzz;
      a.nzc = (g->nz + tzz - 1) / tzz;
      a.ntiles = a.ntx * a.nty * a.nzc * nbatch;
      e.nslots = (long long)a.ntx * a.nty * a.nzc;
      grid = (int)std::max(1LL, std::min((long long)a.ntiles, slots));  // one persistent wave
    }
    if constexpr (WS) kern<<<grid, block, smem, s>>>(mx, mu, mnu, mek, mmask, a, (typename cplx<T>::t*)y, e);
    else kern<<<grid, block, smem, s>>>(mx, my, mu, mnu, mek, mmask, a, e);
    FIT_CHECK_CUDA(cudaGetLastError());
    return FIT_OK;
  };
  if constexpr (WS) {
    switch (e.mode) {
      case FIT_EPI_NONE: return run(ws_apply_kernel<T, TY, FIT_EPI_NONE, S>);
      case FIT_EPI_DOT_U: return run(ws_apply_kernel<T, TY, FIT_EPI_DOT_U, S>);
      case FIT_EPI_DOT_TS: return run(ws_apply_kernel<T, TY, FIT_EPI_DOT_TS, S>);
      case FIT_EPI_RESID: return run(ws_apply_kernel<T, TY, FIT_EPI_RESID, S>);
      case FIT_EPI_DOT_XY: return run(ws_apply_kernel<T, TY, FIT_EPI_DOT_XY, S>);
    }
  } else {
    switch (e.mode) {
      case FIT_EPI_NONE: return run(fused_apply_kernel<T, TY, FIT_EPI_NONE, S>);
      case FIT_EPI_DOT_U: return run(fused_apply_kernel<T, TY, FIT_EPI_DOT_U, S>);
      case FIT_EPI_DOT_TS: return run(fused_apply_kernel<T, TY, FIT_EPI_DOT_TS, S>);
      case FIT_EPI_RESID: return run(fused_apply_kernel<T, TY, FIT_EPI_RESID, S>);
      case FIT_EPI_DOT_XY: return run(fused_apply_kernel<T, TY, FIT_EPI_DOT_XY, S>);
    }
  }
  fit_set_error("fused apply: unknown epilogue");
  return FIT_EINVAL;
}

template <typename T>
fit_status launch_fused(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y, const T* nu,
                        const T* ek, double out_scale, cudaStream_t s, fit_epi& e, const Variant& v) {
#define FIT_LV(TY_, S_, WS_) \
  if (v.ty == TY_ && v.stages == S_ && v.ws == WS_) \
    return launch_variant<T, TY_, S_, WS_>(g, nbatch, omega_dev, x, y, nu, ek, out_scale, s, e, v.tz, v.pf)
  FIT_LV(4, 4, 0);
  FIT_LV(8, 4, 0);
  FIT_LV(16, 3, 0);
  FIT_LV(4, 3, 0);
  FIT_LV(8, 3, 0);
  FIT_LV(4, 4, 1);
  FIT_LV(8, 4, 1);
  if constexpr (sizeof(T) == 4) {  // complex64 only
    FIT_LV(8, 3, 1);
    FIT_LV(16, 4, 1);
    FIT_LV(16, 5, 1);
    FIT_LV(8, 5, 1);
  }
#undef FIT_LV
  fit_set_error("fused apply: no such variant");
  return FIT_EINVAL;
}

const Variant* variants(fit_prec prec, int* n) {
  if (prec == FIT_C64) {
    *n = (int)(sizeof(kVariants64) / sizeof(Variant));
    return kVariants64;
  }
  *n = (int)(sizeof(kVariants128) / sizeof(Variant));
  return kVariants128;
}

// Kernel selection override for tests and experiments: FIT_APPLY_KERNEL=generic forces the generic
// kernel, FIT_APPLY_KERNEL=fused:<k> forces fused variant k.  Returns 0 (automatic), 1 (generic)
// or 2 (fused; *variant set).
int kernel_override(int* variant) {
  const char* s = getenv("FIT_APPLY_KERNEL");
  *variant = 0;
  if (!s) return 0;
  if (!strcmp(s, "generic")) return 1;
  if (!strncmp(s, "fused", 5)) {
    if (s[5] == ':') *variant = atoi(s + 6);
    return 2;
  }
  return 0;
}

bool fused_supported(const fit_grid* g, fit_prec prec) {
  // copies of x start on 16-byte boundaries only if a grid row holds a whole number of 16-byte units
  if (prec == FIT_C64 && (g->nx % 2) != 0) return false;
  return encoder() != nullptr;
}

// dynamic shared memory of variant v with the epilogue vector staged (ku) or not
template <typename T>
int variant_smem(const Variant& v, bool ku) {
#define FIT_SM(TY_, S_, WS_)                                                                              \
  if (v.ty == TY_ && v.stages == S_ && v.ws == WS_)                                                       \
    return (ku ? Layout<T, TY_, true>::smem(S_) : Layout<T, TY_, false>::smem(S_)) +                      \
           (WS_ ? 3 * 8 * S_ + 8 + 8 * 3 * TY_ + 16 : 0)
  FIT_SM(4, 4, 0);
  FIT_SM(8, 4, 0);
  FIT_SM(16, 3, 0);
  FIT_SM(4, 3, 0);
  FIT_SM(8, 3, 0);
  FIT_SM(4, 4, 1);
  FIT_SM(8, 4, 1);
  FIT_SM(8, 3, 1);
  FIT_SM(16, 4, 1);
  FIT_SM(16, 5, 1);
  FIT_SM(8, 5, 1);
#undef FIT_SM
  return 1 << 30;
}

// the variant's shared memory fits one CTA with every epilogue (so an autotuned choice serves them all)
bool fused_smem_ok(fit_prec prec, const Variant& v) {
  const int need = prec == FIT_C64 ? variant_smem<float>(v, true) : variant_smem<double>(v, true);
  return need <= fused_smem_limit();
}

bool fused_fits(const fit_grid* g, int nbatch, const Variant& v) {
  // the persistent loop indexes tiles with int
  const int tz = v.tz > 0 ? v.tz : 2;
  return (long long)((g->nx + TX - 1) / TX) * ((g->ny + v.ty - 1) / v.ty) * ((g->nz + tz - 1) / tz) * nbatch <
         (1LL << 30);
}

}  // namespace

bool fit_tmap_encode(CUtensorMap* m, CUtensorMapDataType dt, int rank, const void* base, const cuuint64_t* dims,
                     const cuuint64_t* strides, const cuuint32_t* box) {
  return encode(m, dt, rank, base, dims, strides, box);
}

fit_status fit_launch_apply_generic(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y,
                                    fit_prec prec, double out_scale, cudaStream_t s, fit_epi* epi);
long long fit_apply_partials_generic(const fit_grid* g);

long long fit_apply_partials(const fit_grid* g, fit_prec prec) {
  long long best = fit_apply_partials_generic(g);
  int n = 0;
  const Variant* v = variants(prec, &n);
  for (int k = 0; k < n; ++k) {
    const int tz = v[k].tz > 0 ? v[k].tz : 2;  // auto chunks are at least 2 planes long
    long long p = (long long)((g->nx + TX - 1) / TX) * ((g->ny + v[k].ty - 1) / v[k].ty) * ((g->nz + tz - 1) / tz);
    best = std::max(best, p);
  }
  return best;
}

static fit_status launch_choice(fit_grid* g, int choice, int nbatch, const double* omega_dev, const void* x, void* y,
                                fit_prec prec, double out_scale, cudaStream_t s, fit_epi& e) {
  if (choice < 0) return fit_launch_apply_generic(g, nbatch, omega_dev, x, y, prec, out_scale, s, &e);
  int n = 0;
  const Variant* v = variants(prec, &n);
  if (choice >= n || !fused_fits(g, nbatch, v[choice]) || !fused_smem_ok(prec, v[choice]))
    return fit_launch_apply_generic(g, nbatch, omega_dev, x, y, prec, out_scale, s, &e);
  if (prec == FIT_C64) return launch_fused<float>(g, nbatch, omega_dev, x, y, g->nu32, g->ek32, out_scale, s, e, v[choice]);
  return launch_fused<double>(g, nbatch, omega_dev, x, y, g->nu64, g->ek64, out_scale, s, e, v[choice]);
}

// Reads a buffer (grid-stride, 16 bytes a thread per step) so that its lines replace whatever the
// L2 held; the store is never taken (the buffer holds 0x01 bytes) but keeps the loads alive.
__global__ void l2_scrub_kernel(const uint4* __restrict__ p, size_t n, uint4* sink) {
  uint4 acc = make_uint4(0u, 0u, 0u, 0u);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint4 v = p[i];
    acc.x ^= v.x;
    acc.y ^= v.y;
    acc.z ^= v.z;
    acc.w ^= v.w;
  }
  if (acc.x == 0xdeadbeefu) *sink = acc;
}

// Autotuner: time every candidate (and the generic kernel) on the caller's buffers, keep the
// fastest per (precision, batch).  Runs on the first apply with a new key outside stream capture.
fit_status fit_tune_apply(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y, fit_prec prec,
                          cudaStream_t s) {
  const long long key = (long long)nbatch * 2 + (prec == FIT_C64 ? 0 : 1);
  if (g->tuned.count(key)) return FIT_OK;
  if (!fused_supported(g, prec)) {
    g->tuned[key] = -1;
    return FIT_OK;
  }
  // opt-in persistence: a cache file named by FIT_TUNE_CACHE supplies the choice for this device, grid,
  // precision and batch if it holds one, and records the result of a new search
  const char* cache = getenv("FIT_TUNE_CACHE");
  std::string dev_name;
  int sms = 0;
  const bool use_cache = cache && *cache && fit_tuning_device_key(&dev_name, &sms) == FIT_OK;
  if (use_cache) {
    int c = -2;
    if (fit_tuning_lookup(cache, dev_name.c_str(), sms, g->nx, g->ny, g->nz, prec, nbatch, &c) == FIT_OK && c >= -1) {
      g->tuned[key] = c;
      return FIT_OK;
    }
  }
  int n = 0;
  const Variant* vars = variants(prec, &n);
  // Candidates are timed from a cold L2, as an apply inside a solve or a sweep mostly runs: before
  // each timed launch half of a scratch buffer of twice the L2 size is written and the other half
  // read, which evicts the operands and leaves only clean lines behind.  Without room for the
  // buffer (HBM budget or memory) the candidates are timed back to back instead.
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  const size_t half = ((size_t)std::max(l2, 1 << 20) + 255) / 256 * 256;
  unsigned char* scratch = nullptr;
  if (!g->budget || g->bytes_held + 2 * half <= g->budget) {
    if (fit_dev_alloc(g, (void**)&scratch, 2 * half) != FIT_OK) scratch = nullptr;
    if (scratch && cudaMemsetAsync(scratch, 1, 2 * half, s) != cudaSuccess) {
      fit_dev_free(g, scratch, 2 * half);
      scratch = nullptr;
    }
  }
  auto cool = [&]() {
    if (!scratch) return;
    cudaMemsetAsync(scratch, 1, half, s);
    l2_scrub_kernel<<<1024, 256, 0, s>>>((const uint4*)(scratch + half), half / 16, (uint4*)scratch);
  };
  cudaEvent_t e0, e1;
  FIT_CHECK_CUDA(cudaEventCreate(&e0));
  FIT_CHECK_CUDA(cudaEventCreate(&e1));
  fit_epi none;
  // three passes over the candidates (so that slow clocks or a neighbour's traffic during one pass
  // do not decide), each candidate timed as the mean of the middle 5 of 7 launches (event times of a
  // single launch come in steps of about 2 us on this part, so a median cannot tell shapes 5% apart);
  // a candidate keeps its best pass
  std::vector<float> t(n + 1, 1e30f);
  for (int pass = 0; pass < 3; ++pass) {
    for (int c = -1; c < n; ++c) {
      if (c >= 0 && (!fused_smem_ok(prec, vars[c]) || !fused_fits(g, nbatch, vars[c]))) continue;
      fit_status st = launch_choice(g, c, nbatch, omega_dev, x, y, prec, 1.0, s, none);  // warm-up
      if (st != FIT_OK) continue;
      float ms[7];
      for (int r = 0; r < 7; ++r) {
        cool();
        cudaEventRecord(e0, s);
        launch_choice(g, c, nbatch, omega_dev, x, y, prec, 1.0, s, none);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        ms[r] = 0.f;
        cudaEventElapsedTime(&ms[r], e0, e1);
      }
      std::sort(ms, ms + 7);
      t[c + 1] = std::min(t[c + 1], (ms[1] + ms[2] + ms[3] + ms[4] + ms[5]) / 5.0f);
    }
  }
  // The fastest candidate wins, except that a shape with an L2 prefetch must beat the fastest shape
  // without one by 2%: the prefetched planes take L2 room that the tuner's scrubbed L2 does not miss but
  // a solve's vectors do, and within 2% the two are not told apart by the tuner's timing (on 128^3 the
  // even split with a 2-plane prefetch timed level with the plain one here and ran 5% slower in the
  // bench's loop).
  float best_ms = 1e30f, best_np_ms = 1e30f;
  int best = -1, best_np = -1;
  for (int c = -1; c < n; ++c) {
    if (t[c + 1] < best_ms) {
      best_ms = t[c + 1];
      best = c;
    }
    if ((c < 0 || vars[c].pf == 0) && t[c + 1] < best_np_ms) {
      best_np_ms = t[c + 1];
      best_np = c;
    }
  }
  if (best != best_np && best_np_ms < 1e29f && best_ms > 0.98f * best_np_ms) {
    best = best_np;
    best_ms = best_np_ms;
  }
  // FIT_TUNE_LOG=1: every candidate's time on stderr (for studying the launch shapes)
  const char* lg = getenv("FIT_TUNE_LOG");
  if (lg && lg[0] == '1') {
    for (int c = -1; c < n; ++c)
      fprintf(stderr, "[fit tune] %dx%dx%d prec %d batch %d: candidate %d %.2f us%s\n", g->nx, g->ny, g->nz, (int)prec,
              nbatch, c, t[c + 1] < 1e29f ? 1e3f * t[c + 1] : -1.f, c == best ? " (chosen)" : "");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (scratch) {
    cudaStreamSynchronize(s);
    fit_dev_free(g, scratch, 2 * half);
  }
  FIT_CHECK_CUDA(cudaGetLastError());
  // kernels that saw the abort word left at once: their times mean nothing, so nothing is cached
  if (fit_check_abort(g, "fit_tune_apply") != FIT_OK) return FIT_ETIMEOUT;
  g->tuned[key] = best;
  if (use_cache)  // a cache that cannot be written leaves the in-memory choice in force
    (void)fit_tuning_record(cache, dev_name.c_str(), sms, g->nx, g->ny, g->nz, prec, nbatch, best);
  return FIT_OK;
}

fit_status fit_launch_apply(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y, fit_prec prec,
                            double out_scale, cudaStream_t s, fit_epi* epi) {
  fit_epi local;
  fit_epi& e = epi ? *epi : local;
  int forced = 0;
  const int ov = kernel_override(&forced);
  const bool aligned = (((uintptr_t)x | (uintptr_t)y) & 15) == 0;
  if (ov == 1 || !aligned || !fused_supported(g, prec))
    return fit_launch_apply_generic(g, nbatch, omega_dev, x, y, prec, out_scale, s, &e);
  if (ov == 2) return launch_choice(g, forced, nbatch, omega_dev, x, y, prec, out_scale, s, e);
  const long long key = (long long)nbatch * 2 + (prec == FIT_C64 ? 0 : 1);
  auto it = g->tuned.find(key);
  if (it == g->tuned.end()) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusNone && epi == nullptr) {
      fit_status st = fit_tune_apply(g, nbatch, omega_dev, x, y, prec, s);
      if (st != FIT_OK) return st;
      it = g->tuned.find(key);
    }
  }
  const int choice = it != g->tuned.end() ? it->second : 0;
  return launch_choice(g, choice, nbatch, omega_dev, x, y, prec, out_scale, s, e);
}

// The apply without the autotuner: the cached choice for (prec, nbatch) if one exists, else the
// first fused variant (or the generic kernel where the fused one does not apply).  Runs no timing,
// creates no events and allocates nothing.
fit_status fit_launch_apply_fixed(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y,
                                  fit_prec prec, double out_scale, cudaStream_t s) {
  fit_epi e;
  const bool aligned = (((uintptr_t)x | (uintptr_t)y) & 15) == 0;
  if (!aligned || !fused_supported(g, prec))
    return fit_launch_apply_generic(g, nbatch, omega_dev, x, y, prec, out_scale, s, &e);
  const long long key = (long long)nbatch * 2 + (prec == FIT_C64 ? 0 : 1);
  auto it = g->tuned.find(key);
  const int choice = it != g->tuned.end() ? it->second : 0;
  return launch_choice(g, choice, nbatch, omega_dev, x, y, prec, out_scale, s, e);
}

int fit_tuned_choice(const fit_grid* g, fit_prec prec, int nbatch, int* out7) {
  const long long key = (long long)nbatch * 2 + (prec == FIT_C64 ? 0 : 1);
  auto it = g->tuned.find(key);
  int c = it == g->tuned.end() ? -2 : it->second;
  out7[0] = c;
  if (c >= 0) {
    int n = 0;
    const Variant* v = variants(prec, &n);
    out7[1] = TX;
    out7[2] = v[c].ty;
    out7[3] = v[c].tz;
    out7[4] = v[c].stages;
    out7[5] = v[c].ws;
    out7[6] = v[c].pf;
  } else {  // the generic kernel: 32 x 8 threads, one plane each
    out7[1] = 32;
    out7[2] = 8;
    out7[3] = 1;
    out7[4] = 0;
    out7[5] = 0;
    out7[6] = 0;
  }
  return c;
}

extern "C" {

int fit_apply_variant_count(fit_prec prec) {
  int n = 0;
  variants(prec, &n);
  return n;
}

fit_status fit_apply_tuned(const fit_grid* g, fit_prec prec, int nbatch, int* out7) {
  FIT_REQUIRE(g && out7 && nbatch >= 1, "fit_apply_tuned: bad argument");
  fit_tuned_choice(g, prec, nbatch, out7);
  return FIT_OK;
}

}  // extern "C"
