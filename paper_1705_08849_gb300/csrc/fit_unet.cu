// Learned right preconditioner: the U-Net runtime (parameters, activations, forward, backward,
// Adam) and its C ABI.  The network maps a normalised complex64 residual plus four material
// channels to a correction: z = rms(v) * U(v / rms(v)) approximates A_in^{-1} v, A_in being the
// scaled complex64 operator of the inner FGMRES.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fit_internal.cuh"
#include "fit_unet_kernels.cuh"

namespace {

enum LayerKind { L_CONV3 = 0, L_TCONV = 1, L_HEAD = 2 };
struct LayerSpec {
  int kind, cin, cout;
};
// c1a c1b | c2a c2b | c3a c3b | t2 c2c c2d | t1 c1c c1d | head
const LayerSpec kLayers[] = {{L_CONV3, 16, 16}, {L_CONV3, 16, 16}, {L_CONV3, 16, 32}, {L_CONV3, 32, 32},
                             {L_CONV3, 32, 64}, {L_CONV3, 64, 64}, {L_TCONV, 64, 32}, {L_CONV3, 64, 32},
                             {L_CONV3, 32, 32}, {L_TCONV, 32, 16}, {L_CONV3, 32, 16}, {L_CONV3, 16, 16},
                             {L_HEAD, 16, 6}};
constexpr int kNL = sizeof(kLayers) / sizeof(kLayers[0]);
enum { C1A, C1B, C2A, C2B, C3A, C3B, T2, C2C, C2D, T1, C1C, C1D, HEAD };

long long wcount(const LayerSpec& l) {
  const long long taps = l.kind == L_CONV3 ? 27 : (l.kind == L_TCONV ? 8 : 1);
  return taps * l.cin * l.cout;
}

unsigned nblocks(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 152LL * 32); }

}  // namespace

struct fit_unet {
  int device = 0;
  long long nparams = 0;
  long long woff[kNL], boff[kNL];
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // master params, grads, Adam moments
  bf16 *wf[kNL] = {}, *wt[kNL] = {};                                // bf16 forward / dgrad conv weights
  double* sums = nullptr;
  int step = 0;
  bool weights_dirty = true;
  // activations for one grid size
  int nx = 0, ny = 0, nz = 0;
  std::vector<std::pair<void*, size_t>> bufs;
  bf16 *A1a, *S1, *P1, *A2a, *S2, *P2, *A3a, *B3, *U2, *A2c, *B2, *U1, *A1c, *B1;
  float *Y, *dY;
  bf16 *g16a, *g16b, *g16c, *g8a, *g8b, *g8c, *g64a, *g64b, *g64c;
  // residual-angle training: complex64 vectors of the grid (z = U's output, w = A z, the normalised
  // residual, a scratch vector), the frequency and the reduction sums on the device
  float2 *rz = nullptr, *rw = nullptr, *rr = nullptr, *rt = nullptr;
  double *rom = nullptr, *rpart = nullptr, *rsum = nullptr;
  long long rne = 0;
  ~fit_unet() {
    for (auto& b : bufs) cudaFree(b.first);
    for (void* q : {(void*)rz, (void*)rw, (void*)rr, (void*)rt, (void*)rom, (void*)rpart, (void*)rsum})
      if (q) cudaFree(q);
    for (int l = 0; l < kNL; ++l) {
      if (wf[l]) cudaFree(wf[l]);
      if (wt[l]) cudaFree(wt[l]);
    }
    cudaFree(p);
    cudaFree(g);
    cudaFree(m);
    cudaFree(v);
    cudaFree(sums);
  }
};

namespace {

fit_status alloc_acts(fit_unet* u, int nx, int ny, int nz) {
  if (u->nx == nx && u->ny == ny && u->nz == nz) return FIT_OK;
  for (auto& b : u->bufs) cudaFree(b.first);
  u->bufs.clear();
  const long long N = (long long)nx * ny * nz, N2 = N / 8, N4 = N / 64;
  auto take = [&](size_t bytes) -> void* {
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, std::max<size_t>(bytes, 256)) != cudaSuccess) return nullptr;
    u->bufs.push_back({ptr, bytes});
    return ptr;
  };
  const size_t b = sizeof(bf16);
  u->A1a = (bf16*)take(N * 16 * b);
  u->S1 = (bf16*)take(N * 16 * b);
  u->P1 = (bf16*)take(N2 * 16 * b);
  u->A2a = (bf16*)take(N2 * 32 * b);
  u->S2 = (bf16*)take(N2 * 32 * b);
  u->P2 = (bf16*)take(N4 * 32 * b);
  u->A3a = (bf16*)take(N4 * 64 * b);
  u->B3 = (bf16*)take(N4 * 64 * b);
  u->U2 = (bf16*)take(N2 * 32 * b);
  u->A2c = (bf16*)take(N2 * 32 * b);
  u->B2 = (bf16*)take(N2 * 32 * b);
  u->U1 = (bf16*)take(N * 16 * b);
  u->A1c = (bf16*)take(N * 16 * b);
  u->B1 = (bf16*)take(N * 16 * b);
  u->Y = (float*)take(N * 6 * sizeof(float));
  u->dY = (float*)take(N * 6 * sizeof(float));
  u->g16a = (bf16*)take(N * 16 * b);
  u->g16b = (bf16*)take(N * 16 * b);
  u->g16c = (bf16*)take(N * 16 * b);
  u->g8a = (bf16*)take(N2 * 32 * b);
  u->g8b = (bf16*)take(N2 * 32 * b);
  u->g8c = (bf16*)take(N2 * 32 * b);
  u->g64a = (bf16*)take(N4 * 64 * b);
  u->g64b = (bf16*)take(N4 * 64 * b);
  u->g64c = (bf16*)take(N4 * 64 * b);
  for (auto& bb : u->bufs)
    if (!bb.first) {
      fit_set_error("U-Net: activation allocation failed");
      return FIT_ENOMEM;
    }
  if (u->bufs.size() != 25) {
    fit_set_error("U-Net: activation allocation failed");
    return FIT_ENOMEM;
  }
  u->nx = nx;
  u->ny = ny;
  u->nz = nz;
  return FIT_OK;
}

void refresh_weights(fit_unet* u, cudaStream_t s) {
  if (!u->weights_dirty) return;
  for (int l = 0; l < kNL; ++l)
    if (kLayers[l].kind == L_CONV3)
      unet::conv_weights_bf16_kernel<<<nblocks(wcount(kLayers[l])), 256, 0, s>>>(
          u->p + u->woff[l], u->wf[l], u->wt[l], kLayers[l].cout, kLayers[l].cin);
  u->weights_dirty = false;
}

// conv3 launch of one (CIN, NC, TY) instantiation: the z-chunk length is chosen so that the
// (x, y, channel-block) columns times the chunks fill the resident CTAs about once
template <int CIN, int NC, int TY>
fit_status launch_conv3(const unet::ConvArgs& a, cudaStream_t s) {
  auto kern = unet::conv3_kernel<CIN, NC, TY>;
  const int smem = unet::Conv3Shape<CIN, NC, TY>::smem();
  static int per_sm = 0, nsm = 0;  // per instantiation, looked up once
  if (per_sm == 0) {
    int dev = 0;
    FIT_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FIT_CHECK_CUDA(cudaGetDevice(&dev));
    FIT_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int p = 0;
    FIT_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, kern, 256, smem));
    if (p < 1) {
      fit_set_error("U-Net: conv tile does not fit on an SM");
      return FIT_EINVAL;
    }
    per_sm = p;
  }
  const int gx = (a.nx + unet::CX - 1) / unet::CX, gy = (a.ny + TY - 1) / TY, nblk = (a.cout + NC - 1) / NC;
  const long long cols = (long long)gx * gy * nblk;
  const long long per_col = std::max(1LL, (long long)per_sm * nsm / cols);
  const int tz = (int)std::max(2LL, ((long long)a.nz + per_col - 1) / per_col);
  const int nzc = (a.nz + tz - 1) / tz;
  dim3 grid(gx, gy, (unsigned)(nzc * nblk));
  kern<<<grid, 256, smem, s>>>(a, tz);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

static bool conv_use_tc();

// tcgen05 transposed conv: persistent CTAs, as many per SM as its TMEM holds accumulators for
template <int CIN, int COUT>
fit_status tconv_fwd_tc(const bf16* in, const float* w, const float* b, bf16* out, int mx, int my, int mz,
                        cudaStream_t s) {
  using SH = unet::TconvTc<CIN, COUT>;
  auto kern = unet::tconv_tc_kernel<CIN, COUT>;
  constexpr int smem = SH::smem();
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    FIT_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FIT_CHECK_CUDA(cudaGetDevice(&dev));
    FIT_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  const long long ntiles = ((long long)mx * my * mz + 127) / 128;
  const int grid = (int)std::min<long long>(ntiles, (long long)nsm * SH::PER_SM);
  kern<<<grid, 128, smem, s>>>(in, w, b, out, mx, my, mz);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

// 2x2x2 transposed conv from an mx x my x mz coarse grid to the 2x finer one
template <int CIN, int COUT>
fit_status tconv_fwd(const bf16* in, const float* w, const float* b, bf16* out, int mx, int my, int mz,
                     cudaStream_t s) {
  if (conv_use_tc()) return tconv_fwd_tc<CIN, COUT>(in, w, b, out, mx, my, mz, s);
  auto kern = unet::tconv_fwd_kernel<CIN, COUT>;
  constexpr int smem = unet::tconv_smem<CIN, COUT>();
  static bool attr = false;
  if (!attr) {
    FIT_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = true;
  }
  const long long n = 8LL * mx * my * mz;
  kern<<<(unsigned)((n + 255) / 256), 256, smem, s>>>(in, w, b, out, mx, my, mz);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

// 5D tensor map {8 channels, C/8 groups, nx, ny, nz} of an NDHWC bf16 activation with C channels,
// box {8, 1, 10, 18, 1}: one channel group of the 10 x 18 voxel window (an 8 x 16 tile and its halo)
// of one plane, the tcgen05 conv's staged layout
static bool conv_tmap(CUtensorMap* m, const bf16* base, int c, int nx, int ny, int nz) {
  const cuuint64_t dims[5] = {8, (cuuint64_t)(c / 8), (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[4] = {16, (cuuint64_t)c * 2, (cuuint64_t)nx * c * 2, (cuuint64_t)nx * ny * c * 2};
  using SH = unet::UmmaShape<16, 16, 4>;
  const cuuint32_t box[5] = {8, 1, (cuuint32_t)SH::PX, (cuuint32_t)SH::PY, 1};
  return fit_tmap_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box);
}

// tcgen05 conv3: 8 x 16 voxel tiles, all output channels per CTA, the same z-chunking rule as
// launch_conv3
template <int CIN, int NC, int S>
fit_status launch_conv3_tc(const unet::ConvArgs& a, cudaStream_t s) {
  auto kern = unet::conv3_tc_kernel<CIN, NC, S>;
  constexpr int smem = unet::UmmaShape<CIN, NC, S>::smem();
  constexpr int TX = unet::UmmaShape<CIN, NC, S>::TX, TY = unet::UmmaShape<CIN, NC, S>::TY;
  // Resident CTAs per SM, from the SM's shared memory (each CTA also reserves 1 KB), its 512 TMEM columns,
  // its 64 K registers and its 2048 threads.  (The runtime's occupancy query answers 1 for this kernel, which left a
  // 128-column grid with one CTA, and one MMA-issuing thread, per SM.)
  static int per_sm = 0, nsm = 0;
  if (per_sm == 0) {
    int dev = 0, smem_sm = 0;
    FIT_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FIT_CHECK_CUDA(cudaGetDevice(&dev));
    FIT_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FIT_CHECK_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    cudaFuncAttributes fa;
    FIT_CHECK_CUDA(cudaFuncGetAttributes(&fa, kern));
    const int by_smem = smem_sm / (smem + 1024), by_tmem = 512 / unet::UmmaShape<CIN, NC, S>::TMEM_COLS;
    const int by_regs = 65536 / (192 * ((fa.numRegs + 7) / 8 * 8));
    const int p = std::min(std::min(by_smem, by_tmem), std::min(by_regs, 2048 / 192));
    if (p < 1) {
      fit_set_error("U-Net: tcgen05 conv tile does not fit on an SM");
      return FIT_EINVAL;
    }
    per_sm = p;
  }
  CUtensorMap m1, m2;
  if (!conv_tmap(&m1, a.in1, a.c1, a.nx, a.ny, a.nz) || (a.c2 > 0 && !conv_tmap(&m2, a.in2, a.c2, a.nx, a.ny, a.nz))) {
    fit_set_error("U-Net: tensor map of a conv input could not be encoded");
    return FIT_ECUDA;
  }
  if (a.c2 == 0) m2 = m1;
  const int gx = (a.nx + TX - 1) / TX, gy = (a.ny + TY - 1) / TY, nblk = (a.cout + NC - 1) / NC;
  const long long cols = (long long)gx * gy * nblk;
  const long long per_col = std::max(1LL, (long long)per_sm * nsm / cols);
  const int tz = (int)std::max(2LL, ((long long)a.nz + per_col - 1) / per_col);
  const int nzc = (a.nz + tz - 1) / tz;
  dim3 grid(gx, gy, (unsigned)(nzc * nblk));
  kern<<<grid, 192, smem, s>>>(m1, m2, a, tz);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

// The convolutions run on the tcgen05 kernels: every 3x3x3 shape (the 64 -> 64 conv in two blocks of 32
// output channels: its 64 x 64 x 27 bf16 weights alone would take 221 KB of shared memory) and both
// transposed convs.  FIT_CONV=mma puts every conv back on the legacy mma.sync / CUDA-core kernels (both paths pass
// the same parity tests; at 128^3 the network takes 0.66 ms on tcgen05 against 1.59 ms on mma.sync).
static bool conv_use_tc() {
  const char* e = getenv("FIT_CONV");
  return !(e && !strcmp(e, "mma"));
}

// the tcgen05 kernel for this shape, if there is one: every channel count a multiple of 8, at most 64
// output channels
static fit_status conv3_tc(const unet::ConvArgs& a, int cin, cudaStream_t s, bool* done) {
  *done = false;
  if (!conv_use_tc() || a.c1 % 8 || a.c2 % 8 || a.o1 % 8 || a.o2 % 8 || a.cout > 64) return FIT_OK;
  // (with cout > NC a CTA computes one block of NC output channels)
  *done = true;
  // shared memory per CTA: weights 27 * cin * NC * 2 B plus S planes of cin / 8 * 2944 B
  if (cin == 16 && a.cout <= 16) return launch_conv3_tc<16, 16, 6>(a, s);  // 50 KB
  if (cin == 16 && a.cout <= 32) return launch_conv3_tc<16, 32, 4>(a, s);  // 52 KB
  if (cin == 16) return launch_conv3_tc<16, 64, 4>(a, s);                  // 79 KB
  if (cin == 32 && a.cout <= 16) return launch_conv3_tc<32, 16, 4>(a, s);  // 76 KB
  if (cin == 32 && a.cout <= 32) return launch_conv3_tc<32, 32, 4>(a, s);  // 103 KB
  if (cin == 32) return launch_conv3_tc<32, 64, 4>(a, s);                  // 159 KB
  if (cin == 64) return launch_conv3_tc<64, 32, 4>(a, s);                  // 206 KB; 64 -> 64 in two blocks
  *done = false;
  return FIT_OK;
}

// Weight gradient of a 3x3x3 conv on the tensor cores: dw (27 x cout x cin) and db accumulate (the caller
// zeroes them); chunks of 1024 voxels per block, 27 taps.
fit_status wgrad_launch(const unet::WgradArgs& w0, cudaStream_t s) {
  unet::WgradArgs w = w0;
  w.chunk = 1024;
  const long long nv = (long long)w.nx * w.ny * w.nz;
  const dim3 grid((unsigned)((nv + w.chunk - 1) / w.chunk), 27);
  const int ci = w.c1 + w.c2, co = w.cout;
#define FIT_WG(CO_, CI_) \
  if (co == CO_ && ci == CI_) { unet::conv3_wgrad_mma_kernel<CO_, CI_><<<grid, 256, 0, s>>>(w); return FIT_OK; }
  FIT_WG(16, 16);
  FIT_WG(32, 16);
  FIT_WG(32, 32);
  FIT_WG(64, 32);
  FIT_WG(64, 64);
  FIT_WG(32, 64);
  FIT_WG(16, 32);
#undef FIT_WG
  fit_set_error("U-Net: unsupported weight-gradient shape");
  return FIT_EINVAL;
}

// conv3 launch: picks the (CIN, NC, TY) instantiation; in2/out2 implement concat / split
fit_status conv3(const bf16* in1, int c1, const bf16* in2, int c2, const bf16* w, const float* bias, bf16* out1, int o1,
                 bf16* out2, int o2, int nx, int ny, int nz, int relu, cudaStream_t s) {
  unet::ConvArgs a;
  a.in1 = in1;
  a.in2 = in2;
  a.c1 = c1;
  a.c2 = c2;
  a.w = w;
  a.bias = bias;
  a.out1 = out1;
  a.out2 = out2;
  a.o1 = o1;
  a.o2 = o2;
  a.cout = o1 + o2;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.relu = relu;
  const int cin = c1 + c2;
  bool done = false;
  const fit_status st = conv3_tc(a, cin, s, &done);
  if (done) return st;
  // shared memory per CTA: (16,16,8) 86 KB, (16,32,8) 107 KB, (32,16,4) 100 KB, (64,16,4) 180 KB
  if (cin == 16 && a.cout <= 16) return launch_conv3<16, 16, 8>(a, s);
  if (cin == 16) return launch_conv3<16, 32, 8>(a, s);
  if (cin == 32) return launch_conv3<32, 16, 4>(a, s);
  if (cin == 64) return launch_conv3<64, 16, 4>(a, s);
  fit_set_error("U-Net: unsupported conv shape");
  return FIT_EINVAL;
}

#define UCK(x)                              \
  do {                                      \
    fit_status st__ = (x);                  \
    if (st__ != FIT_OK) return st__;        \
  } while (0)

fit_status forward(fit_unet* u, const bf16* X0, cudaStream_t s) {
  const int nx = u->nx, ny = u->ny, nz = u->nz;
  const int mx = nx / 2, my = ny / 2, mz = nz / 2, qx = nx / 4, qy = ny / 4, qz = nz / 4;
  const long long N = (long long)nx * ny * nz;
  refresh_weights(u, s);
  auto B = [&](int l) { return u->p + u->boff[l]; };
  UCK(conv3(X0, 16, nullptr, 0, u->wf[C1A], B(C1A), u->A1a, 16, nullptr, 0, nx, ny, nz, 1, s));
  UCK(conv3(u->A1a, 16, nullptr, 0, u->wf[C1B], B(C1B), u->S1, 16, nullptr, 0, nx, ny, nz, 1, s));
  unet::pool_fwd_kernel<<<(unsigned)((N / 8 * 2 + 255) / 256), 256, 0, s>>>(u->S1, u->P1, 16, nx, ny, nz);
  UCK(conv3(u->P1, 16, nullptr, 0, u->wf[C2A], B(C2A), u->A2a, 32, nullptr, 0, mx, my, mz, 1, s));
  UCK(conv3(u->A2a, 32, nullptr, 0, u->wf[C2B], B(C2B), u->S2, 32, nullptr, 0, mx, my, mz, 1, s));
  unet::pool_fwd_kernel<<<(unsigned)((N / 64 * 4 + 255) / 256), 256, 0, s>>>(u->S2, u->P2, 32, mx, my, mz);
  UCK(conv3(u->P2, 32, nullptr, 0, u->wf[C3A], B(C3A), u->A3a, 64, nullptr, 0, qx, qy, qz, 1, s));
  UCK(conv3(u->A3a, 64, nullptr, 0, u->wf[C3B], B(C3B), u->B3, 64, nullptr, 0, qx, qy, qz, 1, s));
  UCK((tconv_fwd<64, 32>(u->B3, u->p + u->woff[T2], B(T2), u->U2, qx, qy, qz, s)));
  UCK(conv3(u->S2, 32, u->U2, 32, u->wf[C2C], B(C2C), u->A2c, 32, nullptr, 0, mx, my, mz, 1, s));
  UCK(conv3(u->A2c, 32, nullptr, 0, u->wf[C2D], B(C2D), u->B2, 32, nullptr, 0, mx, my, mz, 1, s));
  UCK((tconv_fwd<32, 16>(u->B2, u->p + u->woff[T1], B(T1), u->U1, mx, my, mz, s)));
  UCK(conv3(u->S1, 16, u->U1, 16, u->wf[C1C], B(C1C), u->A1c, 16, nullptr, 0, nx, ny, nz, 1, s));
  UCK(conv3(u->A1c, 16, nullptr, 0, u->wf[C1D], B(C1D), u->B1, 16, nullptr, 0, nx, ny, nz, 1, s));
  unet::head_fwd_kernel<16, 6><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(u->B1, u->p + u->woff[HEAD], B(HEAD), u->Y, (int)N);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

// gradient of the loss w.r.t. all parameters into u->g (zeroed here); dY must hold dL/dY
fit_status backward(fit_unet* u, const bf16* X0, cudaStream_t s) {
  const int nx = u->nx, ny = u->ny, nz = u->nz;
  const int mx = nx / 2, my = ny / 2, mz = nz / 2, qx = nx / 4, qy = ny / 4, qz = nz / 4;
  const long long N = (long long)nx * ny * nz, N2 = N / 8, N4 = N / 64;
  FIT_CHECK_CUDA(cudaMemsetAsync(u->g, 0, u->nparams * sizeof(float), s));
  fit_status wg_status = FIT_OK;
  auto GW = [&](int l) { return u->g + u->woff[l]; };
  auto GB = [&](int l) { return u->g + u->boff[l]; };
  auto wgrad = [&](const bf16* dy, int cout, const bf16* x1, int c1, const bf16* x2, int c2, int l, int ax, int ay,
                   int az) {
    unet::WgradArgs w;
    w.dy = dy;
    w.x1 = x1;
    w.x2 = x2;
    w.c1 = c1;
    w.c2 = c2;
    w.cout = cout;
    w.dw = GW(l);
    w.db = GB(l);
    w.nx = ax;
    w.ny = ay;
    w.nz = az;
    if (wgrad_launch(w, s) != FIT_OK) wg_status = FIT_EINVAL;
  };
  auto relu_bwd = [&](bf16* gg, const bf16* y, long long n) { unet::relu_bwd_kernel<<<nblocks(n), 256, 0, s>>>(gg, y, n); };
  // head
  unet::head_bwd_weight_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(u->B1, u->dY, GW(HEAD), GB(HEAD), 16, 6, N);
  unet::head_bwd_data_kernel<<<nblocks(N * 16), 256, 0, s>>>(u->dY, u->p + u->woff[HEAD], u->g16a, 16, 6, N);
  // c1d
  relu_bwd(u->g16a, u->B1, N * 16);
  wgrad(u->g16a, 16, u->A1c, 16, nullptr, 0, C1D, nx, ny, nz);
  UCK(conv3(u->g16a, 16, nullptr, 0, u->wt[C1D], nullptr, u->g16b, 16, nullptr, 0, nx, ny, nz, 0, s));
  // c1c (input S1 ++ U1): d(S1) part -> g16c, d(U1) -> g16a
  relu_bwd(u->g16b, u->A1c, N * 16);
  wgrad(u->g16b, 16, u->S1, 16, u->U1, 16, C1C, nx, ny, nz);
  UCK(conv3(u->g16b, 16, nullptr, 0, u->wt[C1C], nullptr, u->g16c, 16, u->g16a, 16, nx, ny, nz, 0, s));
  // t1: d(B2) -> g8a
  unet::tconv_bwd_weight_kernel<<<dim3((unsigned)((N2 + 127) / 128), 8), 256, 0, s>>>(u->B2, u->g16a, GW(T1), GB(T1), 32,
                                                                                    16, nx, ny, nz, 128);
  unet::tconv_bwd_data_kernel<<<nblocks(N2 * 32), 256, 0, s>>>(u->g16a, u->p + u->woff[T1], u->g8a, 32, 16, nx, ny, nz);
  // c2d
  relu_bwd(u->g8a, u->B2, N2 * 32);
  wgrad(u->g8a, 32, u->A2c, 32, nullptr, 0, C2D, mx, my, mz);
  UCK(conv3(u->g8a, 32, nullptr, 0, u->wt[C2D], nullptr, u->g8b, 32, nullptr, 0, mx, my, mz, 0, s));
  // c2c (input S2 ++ U2): d(S2) part -> g8c, d(U2) -> g8a
  relu_bwd(u->g8b, u->A2c, N2 * 32);
  wgrad(u->g8b, 32, u->S2, 32, u->U2, 32, C2C, mx, my, mz);
  UCK(conv3(u->g8b, 32, nullptr, 0, u->wt[C2C], nullptr, u->g8c, 32, u->g8a, 32, mx, my, mz, 0, s));
  // t2: d(B3) -> g64a
  unet::tconv_bwd_weight_kernel<<<dim3((unsigned)((N4 + 127) / 128), 8), 256, 0, s>>>(u->B3, u->g8a, GW(T2), GB(T2), 64,
                                                                                    32, mx, my, mz, 128);
  unet::tconv_bwd_data_kernel<<<nblocks(N4 * 64), 256, 0, s>>>(u->g8a, u->p + u->woff[T2], u->g64a, 64, 32, mx, my, mz);
  // c3b
  relu_bwd(u->g64a, u->B3, N4 * 64);
  wgrad(u->g64a, 64, u->A3a, 64, nullptr, 0, C3B, qx, qy, qz);
  UCK(conv3(u->g64a, 64, nullptr, 0, u->wt[C3B], nullptr, u->g64b, 64, nullptr, 0, qx, qy, qz, 0, s));
  // c3a (input P2): d(P2) -> g64c (32 channels)
  relu_bwd(u->g64b, u->A3a, N4 * 64);
  wgrad(u->g64b, 64, u->P2, 32, nullptr, 0, C3A, qx, qy, qz);
  UCK(conv3(u->g64b, 64, nullptr, 0, u->wt[C3A], nullptr, u->g64c, 32, nullptr, 0, qx, qy, qz, 0, s));
  // pool2 backward, plus the skip part: d(S2) = g8c + pool_bwd(g64c)
  unet::pool_bwd_kernel<<<nblocks(N2 * 32), 256, 0, s>>>(u->g64c, u->g8a, 32, mx, my, mz);
  unet::bf16_add_kernel<<<nblocks(N2 * 32), 256, 0, s>>>(u->g8c, u->g8a, N2 * 32);
  // c2b
  relu_bwd(u->g8c, u->S2, N2 * 32);
  wgrad(u->g8c, 32, u->A2a, 32, nullptr, 0, C2B, mx, my, mz);
  UCK(conv3(u->g8c, 32, nullptr, 0, u->wt[C2B], nullptr, u->g8b, 32, nullptr, 0, mx, my, mz, 0, s));
  // c2a (input P1): d(P1) -> g8a (16 channels)
  relu_bwd(u->g8b, u->A2a, N2 * 32);
  wgrad(u->g8b, 32, u->P1, 16, nullptr, 0, C2A, mx, my, mz);
  UCK(conv3(u->g8b, 32, nullptr, 0, u->wt[C2A], nullptr, u->g8a, 16, nullptr, 0, mx, my, mz, 0, s));
  // pool1 backward: d(S1) = g16c + pool_bwd(g8a)
  unet::pool_bwd_kernel<<<nblocks(N * 16), 256, 0, s>>>(u->g8a, u->g16a, 16, nx, ny, nz);
  unet::bf16_add_kernel<<<nblocks(N * 16), 256, 0, s>>>(u->g16c, u->g16a, N * 16);
  // c1b
  relu_bwd(u->g16c, u->S1, N * 16);
  wgrad(u->g16c, 16, u->A1a, 16, nullptr, 0, C1B, nx, ny, nz);
  UCK(conv3(u->g16c, 16, nullptr, 0, u->wt[C1B], nullptr, u->g16b, 16, nullptr, 0, nx, ny, nz, 0, s));
  // c1a (input X0; no data gradient needed)
  relu_bwd(u->g16b, u->A1a, N * 16);
  wgrad(u->g16b, 16, X0, 16, nullptr, 0, C1A, nx, ny, nz);
  FIT_CHECK_CUDA(cudaGetLastError());
  return wg_status;
}

fit_status check_dims(int nx, int ny, int nz) {
  if (nx < 4 || ny < 4 || nz < 4 || nx % 4 || ny % 4 || nz % 4) {
    fit_set_error("U-Net: grid dimensions must be multiples of 4 (two 2x poolings)");
    return FIT_EINVAL;
  }
  return FIT_OK;
}

fit_status loss_and_grad(fit_unet* u, const float* target, double* loss, cudaStream_t s) {
  const long long n = (long long)u->nx * u->ny * u->nz * 6;
  FIT_CHECK_CUDA(cudaMemsetAsync(u->sums, 0, 2 * sizeof(double), s));
  unet::loss_sums_kernel<<<nblocks(n), 256, 0, s>>>(u->Y, target, n, u->sums);
  unet::loss_grad_kernel<<<nblocks(n), 256, 0, s>>>(u->Y, target, n, u->sums, u->dY);
  FIT_CHECK_CUDA(cudaGetLastError());
  if (loss) {
    double h[2];
    FIT_CHECK_CUDA(cudaMemcpyAsync(h, u->sums, sizeof(h), cudaMemcpyDeviceToHost, s));
    FIT_CHECK_CUDA(cudaStreamSynchronize(s));
    *loss = h[1] > 0 ? h[0] / h[1] : 0.0;
  }
  return FIT_OK;
}

}  // namespace

// ---- grid-side helpers: input packing and output unpacking --------------------------------------
namespace {

// in16[c][0..5] = scale * (Re, Im) of r_x, r_y, r_z; [6..9] = material channels; [10..15] = 0
__global__ void pack_kernel(const float2* __restrict__ r, float scale, const bf16* __restrict__ mat, bf16* out,
                            long long ncell) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    __align__(16) bf16 v[16];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      const float2 z = r[3 * c + w];
      v[2 * w] = __float2bfloat16(scale * z.x);
      v[2 * w + 1] = __float2bfloat16(scale * z.y);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) v[6 + q] = mat ? mat[4 * c + q] : __float2bfloat16(0.f);
#pragma unroll
    for (int q = 10; q < 16; ++q) v[q] = __float2bfloat16(0.f);
    reinterpret_cast<uint4*>(out + 16 * c)[0] = reinterpret_cast<uint4*>(v)[0];
    reinterpret_cast<uint4*>(out + 16 * c)[1] = reinterpret_cast<uint4*>(v)[1];
  }
}

// z[3c + w] = scale * (y[c][2w] + j y[c][2w+1]) (zero on masked edges) + jac * dinv[3c + w] * v[3c + w]
// when a Jacobi term is given (dinv, v non-null)
__global__ void unpack_kernel(const float* __restrict__ y, float scale, const uint8_t* __restrict__ mask, int nx, int ny,
                              int nxp, float2* z, long long ncell, const float2* __restrict__ dinv,
                              const float2* __restrict__ v, float jac) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    const long long i = c % nx, j = (c / nx) % ny, k = c / ((long long)nx * ny);
    const uint8_t m = mask[i + (long long)nxp * (j + (long long)ny * k)];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      float2 o = ((m >> w) & 1) ? make_float2(0.f, 0.f) : make_float2(scale * y[6 * c + 2 * w], scale * y[6 * c + 2 * w + 1]);
      if (dinv) {
        const float2 d = dinv[3 * c + w], vv = v[3 * c + w];
        o.x += jac * (d.x * vv.x - d.y * vv.y);
        o.y += jac * (d.x * vv.y + d.y * vv.x);
      }
      z[3 * c + w] = o;
    }
  }
}

// t[c][2w..] = scale * (Re, Im) of e[3c + w] (complex128 input), zero on masked edges
__global__ void pack_target_kernel(const double2* __restrict__ e, double scale, const uint8_t* __restrict__ mask, int nx,
                                   int ny, int nxp, float* t, long long ncell) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    const long long i = c % nx, j = (c / nx) % ny, k = c / ((long long)nx * ny);
    const uint8_t m = mask[i + (long long)nxp * (j + (long long)ny * k)];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      const double2 z = ((m >> w) & 1) ? make_double2(0.0, 0.0) : e[3 * c + w];
      t[6 * c + 2 * w] = (float)(scale * z.x);
      t[6 * c + 2 * w + 1] = (float)(scale * z.y);
    }
  }
}

// ---- training pairs ------------------------------------------------------------------------------
// ||xs - xk||^2 (or ||xs||^2 when xk is null) over the unmasked edges, one block, fixed order: out[0]
__global__ void __launch_bounds__(256) pair_err_norm_kernel(const double2* __restrict__ xk, const double2* __restrict__ xs,
                                                            const uint8_t* __restrict__ mask, int nx, int ny, int nxp,
                                                            long long ncell, double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long c = threadIdx.x; c < ncell; c += 256) {
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    const uint8_t m = mask[i + (long long)nxp * (j + (long long)ny * k)];
    for (int w = 0; w < 3; ++w)
      if (!((m >> w) & 1)) {
        const double2 a = xk ? xk[3 * c + w] : make_double2(0.0, 0.0), b = xs[3 * c + w];
        acc += (b.x - a.x) * (b.x - a.x) + (b.y - a.y) * (b.y - a.y);
      }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// pair[c][0..5] = r / rms(r), pair[c][6..11] = (x* - x_k) / rms(x* - x_k), both bf16 and zero on masked
// edges; rms(v) = sqrt(||v||^2 / n_e) with the squared norms in nrm2[0] (residual) and nrm2[1] (error)
__global__ void pair_pack_kernel(const double2* __restrict__ r, const double2* __restrict__ xk,
                                 const double2* __restrict__ xs, const double* __restrict__ nrm2,
                                 const uint8_t* __restrict__ mask, int nx, int ny, int nxp, long long ncell, bf16* pair) {
  const double ne = 3.0 * (double)ncell;
  const double rr2 = nrm2[0] / ne, re2 = nrm2[1] / ne;
  const double ir = rr2 > 0.0 ? 1.0 / sqrt(rr2) : 0.0, ie = re2 > 0.0 ? 1.0 / sqrt(re2) : 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    const uint8_t m = mask[i + (long long)nxp * (j + (long long)ny * k)];
    __align__(16) bf16 v[12];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      double2 in = make_double2(0.0, 0.0), t = make_double2(0.0, 0.0);
      if (!((m >> w) & 1)) {
        const double2 rr = r[3 * c + w], a = xk[3 * c + w], b = xs[3 * c + w];
        in = make_double2(rr.x * ir, rr.y * ir);
        t = make_double2((b.x - a.x) * ie, (b.y - a.y) * ie);
      }
      v[2 * w] = __float2bfloat16((float)in.x);
      v[2 * w + 1] = __float2bfloat16((float)in.y);
      v[6 + 2 * w] = __float2bfloat16((float)t.x);
      v[6 + 2 * w + 1] = __float2bfloat16((float)t.y);
    }
    uint32_t* dst = reinterpret_cast<uint32_t*>(pair + 12 * c);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(v);
#pragma unroll
    for (int q = 0; q < 6; ++q) dst[q] = src[q];
  }
}

// in16[c] = base16[c] with channels 0..5 replaced by the pair's residual channels; target6 = FP32 of the
// pair's target channels
__global__ void pair_sample_kernel(const bf16* __restrict__ pair, const bf16* __restrict__ base16, bf16* in16,
                                   float* target6, long long ncell) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    __align__(16) bf16 v[16];
    *reinterpret_cast<uint4*>(v) = reinterpret_cast<const uint4*>(base16 + 16 * c)[0];
    *reinterpret_cast<uint4*>(v + 8) = reinterpret_cast<const uint4*>(base16 + 16 * c)[1];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      v[q] = pair[12 * c + q];
      target6[6 * c + q] = __bfloat162float(pair[12 * c + 6 + q]);
    }
    reinterpret_cast<uint4*>(in16 + 16 * c)[0] = *reinterpret_cast<uint4*>(v);
    reinterpret_cast<uint4*>(in16 + 16 * c)[1] = *reinterpret_cast<uint4*>(v + 8);
  }
}

// ---- residual-angle loss ------------------------------------------------------------------------
// For a normalised residual r^ (the input's first six channels) and the network's output z (complex64,
// zero on masked edges), with w = A_in z:  L = 1 - |<w, r^>|^2 / (||w||^2 ||r^||^2), the fraction of the
// residual that the direction z cannot remove (flexible GMRES may scale a direction freely).

// r^ from the input's residual channels (bf16), zero on masked edges
__global__ void resid_from_in16_kernel(const bf16* __restrict__ in16, const uint8_t* __restrict__ mask, int nx, int ny,
                                       int nxp, long long ncell, float2* r) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    const long long i = c % nx, j = (c / nx) % ny, k = c / ((long long)nx * ny);
    const uint8_t m = mask[i + (long long)nxp * (j + (long long)ny * k)];
#pragma unroll
    for (int w = 0; w < 3; ++w)
      r[3 * c + w] = ((m >> w) & 1) ? make_float2(0.f, 0.f)
                                    : make_float2(__bfloat162float(in16[16 * c + 2 * w]),
                                                  __bfloat162float(in16[16 * c + 2 * w + 1]));
  }
}

// per-block partials (fixed assignment) of Re, Im <w, r> = sum conj(w) r, ||w||^2 and ||r||^2
__global__ void __launch_bounds__(256) angle_partials_kernel(const float2* __restrict__ w, const float2* __restrict__ r,
                                                             long long n, double* part) {
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
    const float2 a = w[e], b = r[e];
    acc[0] += a.x * b.x + a.y * b.y;
    acc[1] += a.x * b.y - a.y * b.x;
    acc[2] += a.x * a.x + a.y * a.y;
    acc[3] += b.x * b.x + b.y * b.y;
  }
  fit_block_sum<float, 4>(acc, part + 4 * blockIdx.x);
}

// one block: out[0..3] = the fixed-order sums of nb partial slots
__global__ void __launch_bounds__(256) angle_final_kernel(const double* __restrict__ part, int nb, double* out) {
  __shared__ double red[256][4];
  double a[4] = {0, 0, 0, 0};
  for (int q = threadIdx.x; q < nb; q += 256)
    for (int t = 0; t < 4; ++t) a[t] += part[4 * q + t];
  for (int t = 0; t < 4; ++t) red[threadIdx.x][t] = a[t];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int t = 0; t < 4; ++t) red[threadIdx.x][t] += red[threadIdx.x + h][t];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int t = 0; t < 4; ++t) out[t] = red[0][t];
}

// G = dL / d conj(w) = -(conj(c) r - (|c|^2 / n) w) / (n m); writes t = conj(G), so that A t = A conj(G) and
// conj(A t) = conj(A) G = A^H G (A^T = A) is the gradient with respect to conj(z)
__global__ void angle_grad_kernel(const float2* __restrict__ w, const float2* __restrict__ r, const double* __restrict__ sums,
                                  long long n, float2* t) {
  const double cr = sums[0], ci = sums[1], nn = sums[2], mm = sums[3];
  const bool ok = nn > 0.0 && mm > 0.0;
  const float a = ok ? (float)(cr / (nn * mm)) : 0.f, b = ok ? (float)(-ci / (nn * mm)) : 0.f;  // conj(c) / (n m)
  const float q = ok ? (float)((cr * cr + ci * ci) / (nn * nn * mm)) : 0.f;                    // |c|^2 / (n^2 m)
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float2 rv = r[e], wv = w[e];
    const float gx = -(a * rv.x - b * rv.y - q * wv.x), gy = -(a * rv.y + b * rv.x - q * wv.y);
    t[e] = make_float2(gx, -gy);
  }
}

// dL/dY from the gradient conj(A t) with respect to conj(z): dY[c][2w] = 2 Re, dY[c][2w+1] = 2 Im (0 masked)
__global__ void angle_dy_kernel(const float2* __restrict__ at, const uint8_t* __restrict__ mask, int nx, int ny, int nxp,
                                long long ncell, float* dy) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    const long long i = c % nx, j = (c / nx) % ny, k = c / ((long long)nx * ny);
    const uint8_t m = mask[i + (long long)nxp * (j + (long long)ny * k)];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      const float2 g = at[3 * c + w];  // A t = conj(gradient)
      const bool off = (m >> w) & 1;
      dy[6 * c + 2 * w] = off ? 0.f : 2.f * g.x;
      dy[6 * c + 2 * w + 1] = off ? 0.f : -2.f * g.y;
    }
  }
}

}  // namespace

// Used by the solver: z = scale_out * U(scale_in * v) for one complex64 vector (pack, forward,
// unpack); all launches are stream-ordered and capturable.
fit_status fit_unet_apply_vec(fit_unet* u, const fit_grid* g, const void* v, void* z, float scale_in, float scale_out,
                              void* x16, const void* dinv, const void* jac_v, float jac_scale, cudaStream_t s) {
  UCK(check_dims(g->nx, g->ny, g->nz));
  UCK(alloc_acts(u, g->nx, g->ny, g->nz));
  pack_kernel<<<nblocks(g->ncell), 256, 0, s>>>((const float2*)v, scale_in, (const bf16*)g->mat16, (bf16*)x16, g->ncell);
  UCK(forward(u, (const bf16*)x16, s));
  unpack_kernel<<<nblocks(g->ncell), 256, 0, s>>>(u->Y, scale_out, g->mask, g->nx, g->ny, g->nxp, (float2*)z, g->ncell,
                                                  (const float2*)dinv, (const float2*)jac_v, jac_scale);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

int fit_unet_take_timeout() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, unet::g_conv_timeout, sizeof(int)) != cudaSuccess) return 0;
  if (v) {
    const int zero = 0;
    (void)cudaMemcpyToSymbol(unet::g_conv_timeout, &zero, sizeof(int));
  }
  return v;
}

fit_status fit_unet_prepare(fit_unet* u, const fit_grid* g, cudaStream_t s) {
  UCK(check_dims(g->nx, g->ny, g->nz));
  UCK(alloc_acts(u, g->nx, g->ny, g->nz));
  refresh_weights(u, s);  // bf16 weight copies are current before any capture
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

extern "C" {

long long fit_unet_param_count(void) {
  long long n = 0;
  for (int l = 0; l < kNL; ++l) n += wcount(kLayers[l]) + kLayers[l].cout;
  return n;
}

fit_status fit_unet_create(unsigned long long seed, fit_unet** out) {
  FIT_REQUIRE(out, "fit_unet_create: out is NULL");
  *out = nullptr;
  fit_unet* u = new fit_unet();
  FIT_CHECK_CUDA(cudaGetDevice(&u->device));
  long long off = 0;
  for (int l = 0; l < kNL; ++l) {
    u->woff[l] = off;
    off += wcount(kLayers[l]);
    u->boff[l] = off;
    off += kLayers[l].cout;
  }
  u->nparams = off;
  const size_t pb = (size_t)off * sizeof(float);
  if (cudaMalloc(&u->p, pb) || cudaMalloc(&u->g, pb) || cudaMalloc(&u->m, pb) || cudaMalloc(&u->v, pb) ||
      cudaMalloc(&u->sums, 4 * sizeof(double))) {
    delete u;
    fit_set_error("fit_unet_create: allocation failed");
    return FIT_ENOMEM;
  }
  cudaMemset(u->p, 0, pb);
  cudaMemset(u->m, 0, pb);
  cudaMemset(u->v, 0, pb);
  for (int l = 0; l < kNL; ++l) {
    const LayerSpec& L = kLayers[l];
    const double fan_in = (double)(L.kind == L_CONV3 ? 27 : 1) * L.cin;
    // He-normal for the ReLU layers; the head starts at zero, so an untrained network adds nothing
    // to the Jacobi term of the preconditioner
    const double stdv = L.kind == L_CONV3 ? sqrt(2.0 / fan_in) : (L.kind == L_HEAD ? 0.0 : sqrt(1.0 / fan_in));
    unet::init_normal_kernel<<<nblocks(wcount(L)), 256>>>(u->p + u->woff[l], wcount(L), (float)stdv, seed + 7919ULL * l);
    if (L.kind == L_CONV3) {
      const size_t wb = (size_t)wcount(L) * sizeof(bf16);
      if (cudaMalloc(&u->wf[l], wb) || cudaMalloc(&u->wt[l], wb)) {
        delete u;
        fit_set_error("fit_unet_create: allocation failed");
        return FIT_ENOMEM;
      }
    }
  }
  FIT_CHECK_CUDA(cudaDeviceSynchronize());
  *out = u;
  return FIT_OK;
}

void fit_unet_destroy(fit_unet* u) { delete u; }

fit_status fit_unet_get_params(const fit_unet* u, float* host, long long n) {
  FIT_REQUIRE(u && host && n == u->nparams, "fit_unet_get_params: bad argument");
  FIT_CHECK_CUDA(cudaMemcpy(host, u->p, n * sizeof(float), cudaMemcpyDeviceToHost));
  return FIT_OK;
}

fit_status fit_unet_set_params(fit_unet* u, const float* host, long long n) {
  FIT_REQUIRE(u && host && n == u->nparams, "fit_unet_set_params: bad argument");
  FIT_CHECK_CUDA(cudaMemcpy(u->p, host, n * sizeof(float), cudaMemcpyHostToDevice));
  u->weights_dirty = true;
  return FIT_OK;
}

fit_status fit_unet_forward(fit_unet* u, int nx, int ny, int nz, const void* in16, float* out6, void* stream) {
  FIT_REQUIRE(u && in16 && out6, "fit_unet_forward: null argument");
  UCK(check_dims(nx, ny, nz));
  cudaStream_t s = (cudaStream_t)stream;
  UCK(alloc_acts(u, nx, ny, nz));
  UCK(forward(u, (const bf16*)in16, s));
  FIT_CHECK_CUDA(cudaMemcpyAsync(out6, u->Y, (size_t)nx * ny * nz * 6 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return FIT_OK;
}

fit_status fit_unet_backward(fit_unet* u, int nx, int ny, int nz, const void* in16, const float* target6, float* grad,
                             double* loss, void* stream) {
  FIT_REQUIRE(u && in16 && target6, "fit_unet_backward: null argument");
  UCK(check_dims(nx, ny, nz));
  cudaStream_t s = (cudaStream_t)stream;
  UCK(alloc_acts(u, nx, ny, nz));
  UCK(forward(u, (const bf16*)in16, s));
  UCK(loss_and_grad(u, target6, loss, s));
  if (loss && fit_unet_take_timeout()) {  // the loss read-back synchronised the forward pass
    fit_set_error("fit_unet_backward: a bounded wait in a tensor-core convolution ran out");
    return FIT_ETIMEOUT;
  }
  UCK(backward(u, (const bf16*)in16, s));
  if (grad) FIT_CHECK_CUDA(cudaMemcpyAsync(grad, u->g, u->nparams * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return FIT_OK;
}

fit_status fit_unet_train_step(fit_unet* u, int nx, int ny, int nz, const void* in16, const float* target6, float lr,
                               double* loss, void* stream) {
  FIT_REQUIRE(u && in16 && target6 && lr > 0, "fit_unet_train_step: bad argument");
  UCK(fit_unet_backward(u, nx, ny, nz, in16, target6, nullptr, loss, stream));
  cudaStream_t s = (cudaStream_t)stream;
  u->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)u->step), c2 = 1.f - powf(b2, (float)u->step);
  unet::adam_kernel<<<nblocks(u->nparams), 256, 0, s>>>(u->p, u->g, u->m, u->v, u->nparams, lr, b1, b2, 1e-8f, c1, c2);
  FIT_CHECK_CUDA(cudaGetLastError());
  u->weights_dirty = true;
  return FIT_OK;
}

fit_status fit_unet_pack(const fit_grid* g, const void* r, double scale, void* out16, void* stream) {
  FIT_REQUIRE(g && r && out16, "fit_unet_pack: null argument");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  pack_kernel<<<nblocks(g->ncell), 256, 0, (cudaStream_t)stream>>>((const float2*)r, (float)scale,
                                                                    (const bf16*)g->mat16, (bf16*)out16, g->ncell);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

fit_status fit_unet_pack_target(const fit_grid* g, const void* e, double scale, float* out6, void* stream) {
  FIT_REQUIRE(g && e && out6, "fit_unet_pack_target: null argument");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  pack_target_kernel<<<nblocks(g->ncell), 256, 0, (cudaStream_t)stream>>>((const double2*)e, scale, g->mask, g->nx,
                                                                           g->ny, g->nxp, out6, g->ncell);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

fit_status fit_unet_unpack(const fit_grid* g, const float* y6, double scale, void* z, void* stream) {
  FIT_REQUIRE(g && y6 && z, "fit_unet_unpack: null argument");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  unpack_kernel<<<nblocks(g->ncell), 256, 0, (cudaStream_t)stream>>>(y6, (float)scale, g->mask, g->nx, g->ny, g->nxp,
                                                                      (float2*)z, g->ncell, nullptr, nullptr, 0.f);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

// ---- single layers (the kernels the network runs, one at a time) ---------------------------------
namespace {
bool conv_shape_ok(int cin, int cout) {  // the 3x3x3 layer shapes of the network
  static const int ok[][2] = {{16, 16}, {16, 32}, {32, 32}, {32, 64}, {64, 64}, {64, 32}, {32, 16}};
  for (auto& p : ok)
    if (p[0] == cin && p[1] == cout) return true;
  return false;
}
// bf16 forward copy W[tap][co][ci] and dgrad copy W[26 - tap][ci][co] of FP32 weights, in stream-ordered
// scratch that the caller frees with cudaFreeAsync
fit_status layer_weights(const float* w, int cin, int cout, bf16** wf, bf16** wt, cudaStream_t s) {
  const size_t wb = (size_t)27 * cin * cout * sizeof(bf16);
  FIT_CHECK_CUDA(cudaMallocAsync((void**)wf, wb, s));
  FIT_CHECK_CUDA(cudaMallocAsync((void**)wt, wb, s));
  unet::conv_weights_bf16_kernel<<<nblocks(27LL * cin * cout), 256, 0, s>>>(w, *wf, *wt, cout, cin);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}
}  // namespace

fit_status fit_unet_conv3(int nx, int ny, int nz, int cin, int cout, const void* in, const float* w, const float* bias,
                          int relu, void* out, void* stream) {
  FIT_REQUIRE(in && w && out && nx >= 1 && ny >= 1 && nz >= 1, "fit_unet_conv3: bad argument");
  FIT_REQUIRE(conv_shape_ok(cin, cout), "fit_unet_conv3: (cin, cout) is not a layer shape of the network");
  cudaStream_t s = (cudaStream_t)stream;
  bf16 *wf = nullptr, *wt = nullptr;
  UCK(layer_weights(w, cin, cout, &wf, &wt, s));
  fit_status st = conv3((const bf16*)in, cin, nullptr, 0, wf, bias, (bf16*)out, cout, nullptr, 0, nx, ny, nz,
                        relu ? 1 : 0, s);
  cudaFreeAsync(wf, s);
  cudaFreeAsync(wt, s);
  return st;
}

fit_status fit_unet_conv3_dgrad(int nx, int ny, int nz, int cin, int cout, const void* dout, const float* w, void* din,
                                void* stream) {
  FIT_REQUIRE(dout && w && din && nx >= 1 && ny >= 1 && nz >= 1, "fit_unet_conv3_dgrad: bad argument");
  FIT_REQUIRE(conv_shape_ok(cin, cout), "fit_unet_conv3_dgrad: (cin, cout) is not a layer shape of the network");
  cudaStream_t s = (cudaStream_t)stream;
  bf16 *wf = nullptr, *wt = nullptr;
  UCK(layer_weights(w, cin, cout, &wf, &wt, s));
  fit_status st = conv3((const bf16*)dout, cout, nullptr, 0, wt, nullptr, (bf16*)din, cin, nullptr, 0, nx, ny, nz, 0, s);
  cudaFreeAsync(wf, s);
  cudaFreeAsync(wt, s);
  return st;
}

fit_status fit_unet_conv3_wgrad(int nx, int ny, int nz, int cin, int cout, const void* in, const void* dout, float* dw,
                                float* db, void* stream) {
  FIT_REQUIRE(in && dout && dw && nx >= 1 && ny >= 1 && nz >= 1, "fit_unet_conv3_wgrad: bad argument");
  FIT_REQUIRE(conv_shape_ok(cin, cout), "fit_unet_conv3_wgrad: (cin, cout) is not a layer shape of the network");
  cudaStream_t s = (cudaStream_t)stream;
  FIT_CHECK_CUDA(cudaMemsetAsync(dw, 0, (size_t)27 * cin * cout * sizeof(float), s));
  if (db) FIT_CHECK_CUDA(cudaMemsetAsync(db, 0, (size_t)cout * sizeof(float), s));
  unet::WgradArgs a;
  a.dy = (const bf16*)dout;
  a.x1 = (const bf16*)in;
  a.x2 = nullptr;
  a.c1 = cin;
  a.c2 = 0;
  a.cout = cout;
  a.dw = dw;
  a.db = db;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  UCK(wgrad_launch(a, s));
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

fit_status fit_unet_tconv(int mx, int my, int mz, int cin, int cout, const void* in, const float* w, const float* b,
                          void* out, void* stream) {
  FIT_REQUIRE(in && w && b && out && mx >= 1 && my >= 1 && mz >= 1, "fit_unet_tconv: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (cin == 64 && cout == 32) return tconv_fwd<64, 32>((const bf16*)in, w, b, (bf16*)out, mx, my, mz, s);
  if (cin == 32 && cout == 16) return tconv_fwd<32, 16>((const bf16*)in, w, b, (bf16*)out, mx, my, mz, s);
  fit_set_error("fit_unet_tconv: (cin, cout) must be (64, 32) or (32, 16)");
  return FIT_EINVAL;
}

fit_status fit_unet_tconv_backward(int mx, int my, int mz, int cin, int cout, const void* in, const void* dout,
                                   const float* w, void* din, float* dw, float* db, void* stream) {
  FIT_REQUIRE(in && dout && w && din && dw && db && mx >= 1 && my >= 1 && mz >= 1,
              "fit_unet_tconv_backward: bad argument");
  FIT_REQUIRE((cin == 64 && cout == 32) || (cin == 32 && cout == 16),
              "fit_unet_tconv_backward: (cin, cout) must be (64, 32) or (32, 16)");
  cudaStream_t s = (cudaStream_t)stream;
  const int nx = 2 * mx, ny = 2 * my, nz = 2 * mz;
  const long long nc = (long long)mx * my * mz;
  FIT_CHECK_CUDA(cudaMemsetAsync(dw, 0, (size_t)8 * cin * cout * sizeof(float), s));
  FIT_CHECK_CUDA(cudaMemsetAsync(db, 0, (size_t)cout * sizeof(float), s));
  unet::tconv_bwd_data_kernel<<<nblocks(nc * cin), 256, 0, s>>>((const bf16*)dout, w, (bf16*)din, cin, cout, nx, ny, nz);
  unet::tconv_bwd_weight_kernel<<<dim3((unsigned)((nc + 127) / 128), 8), 256, 0, s>>>(
      (const bf16*)in, (const bf16*)dout, dw, db, cin, cout, nx, ny, nz, 128);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

fit_status fit_unet_head(long long nvox, const void* in, const float* w, const float* b, float* out, void* stream) {
  FIT_REQUIRE(in && w && b && out && nvox >= 1 && nvox < (1LL << 31), "fit_unet_head: bad argument");
  unet::head_fwd_kernel<16, 6><<<(unsigned)((nvox + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      (const bf16*)in, w, b, out, (int)nvox);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

fit_status fit_unet_head_backward(long long nvox, const void* in, const float* dout, const float* w, void* din,
                                  float* dw, float* db, void* stream) {
  FIT_REQUIRE(in && dout && w && din && dw && db && nvox >= 1, "fit_unet_head_backward: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  FIT_CHECK_CUDA(cudaMemsetAsync(dw, 0, 6 * 16 * sizeof(float), s));
  FIT_CHECK_CUDA(cudaMemsetAsync(db, 0, 6 * sizeof(float), s));
  unet::head_bwd_weight_kernel<<<(unsigned)((nvox + 255) / 256), 256, 0, s>>>((const bf16*)in, dout, dw, db, 16, 6,
                                                                              nvox);
  unet::head_bwd_data_kernel<<<nblocks(nvox * 16), 256, 0, s>>>(dout, w, (bf16*)din, 16, 6, nvox);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

fit_status fit_unet_training_pair(fit_grid* g, double omega, const void* xk, const void* xstar, const void* b,
                                  void* pair, double* rms_out, void* stream) {
  FIT_REQUIRE(g && xk && xstar && b && pair, "fit_unet_training_pair: null argument");
  FIT_REQUIRE(g->has_materials, "fit_unet_training_pair: materials not set");
  FIT_REQUIRE(isfinite(omega), "fit_unet_training_pair: omega must be finite");
  FIT_REQUIRE((((uintptr_t)pair) & 3) == 0, "fit_unet_training_pair: pair must be 4-byte aligned");
  if (fit_check_abort(g, "fit_unet_training_pair") != FIT_OK) return FIT_ETIMEOUT;
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = (cudaStream_t)stream;
  FitDevTmp tmp(g);
  void *d_om = nullptr, *r = nullptr, *part = nullptr, *nrm = nullptr;
  const long long nslots = fit_apply_partials(g, FIT_C128);
  fit_status st;
  if ((st = tmp.copy(&d_om, &omega, sizeof(double), s)) != FIT_OK) return st;
  if ((st = tmp.alloc(&r, (size_t)g->ne * sizeof(double2))) != FIT_OK) return st;
  if ((st = tmp.alloc(&part, (size_t)nslots * 4 * sizeof(double))) != FIT_OK) return st;
  if ((st = tmp.alloc(&nrm, 2 * sizeof(double))) != FIT_OK) return st;
  // r = b - A x_k in FP64 (the residual epilogue; its norm partials are not used: the norms below skip the
  // masked edges)
  fit_epi e;
  e.mode = FIT_EPI_RESID;
  e.u = b;
  e.part = (double*)part;
  if ((st = fit_launch_apply(g, 1, (const double*)d_om, xk, r, FIT_C128, 1.0, s, &e)) != FIT_OK) return st;
  if (e.nslots > nslots) {
    fit_set_error("fit_unet_training_pair: the apply wrote more partial slots than were allocated");
    return FIT_ECUDA;
  }
  pair_err_norm_kernel<<<1, 256, 0, s>>>(nullptr, (const double2*)r, g->mask, g->nx, g->ny, g->nxp, g->ncell,
                                         (double*)nrm);
  pair_err_norm_kernel<<<1, 256, 0, s>>>((const double2*)xk, (const double2*)xstar, g->mask, g->nx, g->ny, g->nxp,
                                         g->ncell, (double*)nrm + 1);
  pair_pack_kernel<<<nblocks(g->ncell), 256, 0, s>>>((const double2*)r, (const double2*)xk, (const double2*)xstar,
                                                     (const double*)nrm, g->mask, g->nx, g->ny, g->nxp, g->ncell,
                                                     (bf16*)pair);
  FIT_CHECK_CUDA(cudaGetLastError());
  double n2 = 0.0;
  FIT_CHECK_CUDA(cudaMemcpyAsync(&n2, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
  FIT_CHECK_CUDA(cudaStreamSynchronize(s));  // the temporaries are freed on return
  if (rms_out) *rms_out = sqrt(n2 / (double)g->ne);  // rms(r) over the unmasked edges
  return fit_take_device_error(g);
}

fit_status fit_unet_pair_sample(long long ncell, const void* pair, const void* base16, void* in16, float* target6,
                                void* stream) {
  FIT_REQUIRE(pair && base16 && in16 && target6 && ncell >= 1, "fit_unet_pair_sample: bad argument");
  FIT_REQUIRE(((((uintptr_t)base16) | ((uintptr_t)in16)) & 15) == 0,
              "fit_unet_pair_sample: base16 and in16 must be 16-byte aligned");
  pair_sample_kernel<<<nblocks(ncell), 256, 0, (cudaStream_t)stream>>>((const bf16*)pair, (const bf16*)base16,
                                                                        (bf16*)in16, target6, ncell);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

namespace {
constexpr int kAngleBlocks = 608;  // partial slots of the residual-angle sums (4 per SM)

// forward, z = unpack(Y), w = A_in z, r^ from the input, and the four sums; the loss on the host
fit_status angle_forward(fit_unet* u, fit_grid* g, double omega, const bf16* in16, double* loss, cudaStream_t s) {
  UCK(check_dims(g->nx, g->ny, g->nz));
  UCK(alloc_acts(u, g->nx, g->ny, g->nz));
  if (u->rne != g->ne) {
    for (void* q : {(void*)u->rz, (void*)u->rw, (void*)u->rr, (void*)u->rt}) if (q) cudaFree(q);
    u->rz = u->rw = u->rr = u->rt = nullptr;
    const size_t vb = (size_t)g->ne * sizeof(float2);
    if (cudaMalloc(&u->rz, vb) || cudaMalloc(&u->rw, vb) || cudaMalloc(&u->rr, vb) || cudaMalloc(&u->rt, vb)) {
      fit_set_error("fit_unet_train_step_residual: allocation failed");
      u->rne = 0;
      return FIT_ENOMEM;
    }
    u->rne = g->ne;
  }
  if (!u->rom && (cudaMalloc(&u->rom, sizeof(double)) || cudaMalloc(&u->rpart, 4 * kAngleBlocks * sizeof(double)) ||
                  cudaMalloc(&u->rsum, 4 * sizeof(double)))) {
    fit_set_error("fit_unet_train_step_residual: allocation failed");
    return FIT_ENOMEM;
  }
  FIT_CHECK_CUDA(cudaMemcpyAsync(u->rom, &omega, sizeof(double), cudaMemcpyHostToDevice, s));
  UCK(forward(u, in16, s));
  unpack_kernel<<<nblocks(g->ncell), 256, 0, s>>>(u->Y, 1.f, g->mask, g->nx, g->ny, g->nxp, u->rz, g->ncell, nullptr,
                                                  nullptr, 0.f);
  resid_from_in16_kernel<<<nblocks(g->ncell), 256, 0, s>>>(in16, g->mask, g->nx, g->ny, g->nxp, g->ncell, u->rr);
  UCK(fit_launch_apply(g, 1, u->rom, u->rz, u->rw, FIT_C64, 1.0, s));  // the scaled operator A_in
  angle_partials_kernel<<<kAngleBlocks, 256, 0, s>>>(u->rw, u->rr, g->ne, u->rpart);
  angle_final_kernel<<<1, 256, 0, s>>>(u->rpart, kAngleBlocks, u->rsum);
  FIT_CHECK_CUDA(cudaGetLastError());
  if (loss) {
    double h[4];
    FIT_CHECK_CUDA(cudaMemcpyAsync(h, u->rsum, sizeof(h), cudaMemcpyDeviceToHost, s));
    FIT_CHECK_CUDA(cudaStreamSynchronize(s));
    *loss = (h[2] > 0 && h[3] > 0) ? 1.0 - (h[0] * h[0] + h[1] * h[1]) / (h[2] * h[3]) : 1.0;
  }
  return FIT_OK;
}
}  // namespace

fit_status fit_unet_residual_loss(fit_unet* u, fit_grid* g, double omega, const void* in16, double* loss, void* stream) {
  FIT_REQUIRE(u && g && in16 && loss, "fit_unet_residual_loss: null argument");
  FIT_REQUIRE(g->has_materials && isfinite(omega), "fit_unet_residual_loss: materials not set or bad omega");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  return angle_forward(u, g, omega, (const bf16*)in16, loss, (cudaStream_t)stream);
}

fit_status fit_unet_train_step_residual(fit_unet* u, fit_grid* g, double omega, const void* in16, float lr,
                                        double* loss, void* stream) {
  FIT_REQUIRE(u && g && in16 && lr > 0, "fit_unet_train_step_residual: bad argument");
  FIT_REQUIRE(g->has_materials && isfinite(omega), "fit_unet_train_step_residual: materials not set or bad omega");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = (cudaStream_t)stream;
  UCK(angle_forward(u, g, omega, (const bf16*)in16, loss, s));
  // dL/dY: conj(A conj(G)) with G the gradient with respect to conj(w)
  angle_grad_kernel<<<nblocks(g->ne), 256, 0, s>>>(u->rw, u->rr, u->rsum, g->ne, u->rt);
  UCK(fit_launch_apply(g, 1, u->rom, u->rt, u->rw, FIT_C64, 1.0, s));
  angle_dy_kernel<<<nblocks(g->ncell), 256, 0, s>>>(u->rw, g->mask, g->nx, g->ny, g->nxp, g->ncell, u->dY);
  UCK(backward(u, (const bf16*)in16, s));
  u->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)u->step), c2 = 1.f - powf(b2, (float)u->step);
  unet::adam_kernel<<<nblocks(u->nparams), 256, 0, s>>>(u->p, u->g, u->m, u->v, u->nparams, lr, b1, b2, 1e-8f, c1, c2);
  FIT_CHECK_CUDA(cudaGetLastError());
  u->weights_dirty = true;
  return FIT_OK;
}

fit_status fit_set_preconditioner(fit_grid* g, int kind, fit_unet* net) {
  FIT_REQUIRE(g, "fit_set_preconditioner: null grid");
  FIT_REQUIRE(kind == FIT_PC_UNET, "fit_set_preconditioner: only FIT_PC_UNET takes a network");
  g->unet = net;
  return FIT_OK;
}

}  // extern "C"
