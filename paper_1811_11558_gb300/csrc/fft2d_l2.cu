// Whole-plane 2-D real FFTs in one kernel pass (FP32), the row spectra exchanged through L2.
//
// One thread-block cluster of CL CTAs per (layer, component) plane of the Sec. 3.1
// discrete Fourier transform.
//
// Forward (plastic-strain plane -> half spectrum):
//   row phase     CTA r transforms rows x2 in [r R, (r+1) R) (R = N2 / CL), two real rows
//                 per complex FFT, splits the Hermitian pairs and writes the half rows
//                 k1 < N1/2 straight into the spectrum buffer (the k1 = N1/2 coefficient, real
//                 for a real row, goes to the side array nq);
//   cluster barrier (release / acquire at cluster scope: every row of the plane is written);
//   column phase  CTA r transforms the columns k1 in [r H1/CL, (r+1) H1/CL) in place, reading
//                 them with L1-bypassing loads.
// Inverse (half spectrum -> real plane): the column phase first (in place), the barrier,
//   then the rows (Hermitian rebuild, inverse complex FFT, two real rows per transform).
//
// The intermediate row spectra are written and read back within one cluster's lifetime, so
// they are served by L2 and, as long as they stay there, each plane crosses HBM once per
// direction: 8 B per voxel read + 8 B written, against twice that for separate row and column
// kernels.  Unlike the distributed-shared-memory variant (fft2d_cluster.cu) a CTA keeps only
// its FFT exchange area in shared memory, so two CTAs of 512 threads fit on an SM and the
// load, transform and store phases of different clusters overlap.
//
// Hooke's law is not applied here (C:eps_p needs the six components of a voxel, which sit in
// six planes): the depth kernel applies it per mode, and the inverse applies it to the
// k1 = N1/2 column of the stress output.
#include <cooperative_groups.h>

#include "fvim_internal.cuh"

namespace cg = cooperative_groups;

namespace {

// FFT groups of length-N register transforms: N/8 threads per transform, whole warps per
// group (a warp holds two length-128 transforms), FPG transforms per group
template <int N> struct Grp {
  static constexpr int T8 = N / 8;
  static constexpr int NG = T8 < 32 ? 32 : T8;
  static constexpr int FPG = NG / T8;
  static constexpr int LD = N + N / 8;  // padded exchange stride of one transform (complex)
};

// NT threads per CTA (256: three CTAs per SM, at most 85 registers)
template <int NT> struct MinBlocks { static constexpr int v = NT == 256 ? 3 : 2; };

template <int N1, int N2, int CL, int NT> struct Pl {
  typedef Grp<N1> GR_;
  typedef Grp<N2> GC_;
  static constexpr int H1 = N1 / 2;
  static constexpr int RPC = N2 / CL;           // real rows per CTA
  static constexpr int CPC = H1 / CL;           // k1 columns per CTA
  static constexpr int GR = NT / GR_::NG;       // row groups
  static constexpr int RU = 2 * GR_::FPG;       // real rows per row unit (two per transform)
  static constexpr int NRU = RPC / RU;          // row units per CTA
  static constexpr int GC = NT / GC_::NG;       // column groups
  static constexpr int CU = 2 * GC_::FPG;       // columns per column unit (two per transform)
  static constexpr int NCU = CPC / CU;          // column units per CTA
  static constexpr size_t mx(size_t a, size_t b) { return a > b ? a : b; }
  // one pipeline stage of a group: the unit's staged input, then (after it is read into
  // registers) the exchange area of the unit's transforms
  static constexpr size_t ROW_STAGE = mx(mx((size_t)RU * N1 * sizeof(float), (size_t)RU * H1 * sizeof(float2)),
                                         (size_t)GR_::FPG * GR_::LD * sizeof(float2));
  // column passes: every group takes CU adjacent columns, the CTA CPP = GC CU adjacent columns
  // per pass (one 16-byte column pair per row and thread); a pair's region holds its staged
  // rows, then its two transforms' exchange
  static constexpr int NP = GC * GC_::FPG;      // column pairs per pass
  static constexpr int CPP = 2 * NP;            // columns per pass
  static constexpr int NCP = CPC / CPP;         // column passes per CTA
  static constexpr size_t PAIR = mx((size_t)N2 * 2, (size_t)2 * GC_::LD) * sizeof(float2) + 16;
  static constexpr size_t COL_STAGE = (size_t)NP * PAIR;
  static constexpr size_t SMEM = mx((size_t)GR * 2 * ROW_STAGE, 2 * COL_STAGE);
  static_assert(N1 >= 64 && N2 >= 64, "register FFTs of at least 8 threads");
  static_assert(GR >= 1 && GC >= 1 && GR * GR_::NG == NT && GC * GC_::NG == NT, "thread split");
  static_assert(GR <= 15 && GC <= 15, "named barriers 1..15");
  static_assert(RPC % RU == 0 && CPC % CPP == 0 && NRU >= 1 && NCP >= 1, "whole units per CTA");
  static_assert(ROW_STAGE % 16 == 0 && PAIR % 16 == 0, "16-byte stages");
  static_assert(SMEM * MinBlocks<NT>::v <= 227 * 1024, "resident CTAs per SM");
};

// padded exchange of the transforms of one stage: transform f at buf[f LD + p + p/8]
template <int LD> struct PadX {
  float2* buf;
  __device__ __forceinline__ void put(int f, int p, float2 x) const { buf[f * LD + p + (p >> 3)] = x; }
  __device__ __forceinline__ float2 get(int f, int p) const { return buf[f * LD + p + (p >> 3)]; }
};

// column phase of one plane, in place: the CTA's k1 range [kb0, kb0 + CPC) in passes of CPP
// adjacent columns.  Each pass is staged with 16-byte L1-bypassing copies (CPP x 8 bytes of
// every row, consecutive threads on consecutive column pairs) while the previous one is
// transformed; a thread owns one column pair (two transforms, v[0] and v[1]) of its group;
// the results leave through the same staging area with the same row segments.
template <int N1, int N2, int CL, int NT, bool INV>
__device__ __forceinline__ void column_phase(float2* __restrict__ P, int kb0, unsigned char* sm,
                                             const float2* __restrict__ tw2) {
  typedef Pl<N1, N2, CL, NT> Q;
  typedef typename Q::GC_ G;
  constexpr int US = (int)(Q::PAIR / sizeof(float2));  // pair region stride (complex)
  const int g = threadIdx.x / G::NG, lane = threadIdx.x % G::NG;
  const int jp = g * G::FPG + lane / G::T8;  // column pair of the pass owned by this thread
  const int t = lane % G::T8;
  const GroupSync<G::NG> gsync{1 + g};
  float2* st[2] = {reinterpret_cast<float2*>(sm), reinterpret_cast<float2*>(sm + Q::COL_STAGE)};
  auto issue = [&](int pc, float2* dst) {
    const int kb = kb0 + pc * Q::CPP;
    for (int i = threadIdx.x; i < N2 * Q::NP; i += NT) {
      const int row = i / Q::NP, q = i - row * Q::NP;
      cp_async_16(dst + q * US + 2 * row, P + (size_t)row * Q::H1 + kb + 2 * q);
    }
    cp_async_commit();
  };
  issue(0, st[0]);
#pragma unroll 1
  for (int pc = 0; pc < Q::NCP; ++pc) {
    float2* cur = st[pc & 1];
    if (pc + 1 < Q::NCP) {
      __syncthreads();  // pass pc - 1 is done with the buffer the next pass is staged into
      issue(pc + 1, st[(pc + 1) & 1]);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // pass pc's copies of every thread have landed
    float2* reg = cur + jp * US;
    float2 v[2][8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const float4 a = *reinterpret_cast<const float4*>(reg + 2 * (t + m * G::T8));
      v[0][m] = make_float2(a.x, a.y);
      v[1][m] = make_float2(a.z, a.w);
    }
    gsync();  // the pair's region is free: it becomes its transforms' exchange area
    PadX<G::LD> x{reg};
    fft_ct<float2, INV, N2, 2, 1>(v, t, x, tw2, gsync);
    // results back into the pair's region as [row][2], then out with the pass's row segments
    // whole (consecutive threads on consecutive column pairs of a row)
#pragma unroll
    for (int m = 0; m < 8; ++m)
      *reinterpret_cast<float4*>(reg + 2 * (t + m * G::T8)) = make_float4(v[0][m].x, v[0][m].y, v[1][m].x, v[1][m].y);
    __syncthreads();
    const int kb = kb0 + pc * Q::CPP;
    for (int i = threadIdx.x; i < N2 * Q::NP; i += NT) {
      const int row = i / Q::NP, q = i - row * Q::NP;
      *reinterpret_cast<float4*>(P + (size_t)row * Q::H1 + kb + 2 * q) =
          *reinterpret_cast<const float4*>(cur + q * US + 2 * row);
    }
  }
}

template <int N1, int N2, int CL, int NT>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT, MinBlocks<NT>::v)
    k_fft2f_l2(const float* __restrict__ src, float2* __restrict__ spec, float* __restrict__ nq,
               const float2* __restrict__ tw1, const float2* __restrict__ tw2, const int* __restrict__ zr) {
  typedef Pl<N1, N2, CL, NT> Q;
  typedef typename Q::GR_ G;
  extern __shared__ __align__(16) unsigned char smraw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const size_t pl = blockIdx.y;
  if (zr && ((int)(pl / 6) < zr[0] || (int)(pl / 6) >= zr[1])) return;  // layer without input (whole cluster)
  float2* P = spec + pl * (size_t)N2 * Q::H1;

  // 1. row phase: group g transforms row units g, g + GR, ... (RU rows each, one contiguous
  //    block of the plane), staging the next unit while it transforms the current one
  {
    const int g = threadIdx.x / G::NG, lane = threadIdx.x % G::NG;
    const int j = lane / G::T8, t = lane % G::T8;  // transform of the unit, thread within it
    const GroupSync<G::NG> gsync{1 + g};
    unsigned char* st[2] = {smraw + (size_t)(2 * g) * Q::ROW_STAGE, smraw + (size_t)(2 * g + 1) * Q::ROW_STAGE};
    const float* blk0 = src + (pl * N2 + (size_t)r * Q::RPC) * N1;
    auto issue = [&](int u, unsigned char* dst) {
      const float* s = blk0 + (size_t)u * Q::RU * N1;
      float* d = reinterpret_cast<float*>(dst);
      for (int i = lane; i < Q::RU * N1 / 4; i += G::NG) cp_async_16(d + 4 * i, s + 4 * i);
      cp_async_commit();
    };
    if (g < Q::NRU) issue(g, st[0]);
#pragma unroll 1
    for (int it = 0, u = g; u < Q::NRU; ++it, u += Q::GR) {
      unsigned char* cur = st[it & 1];
      if (u + Q::GR < Q::NRU) {
        issue(u + Q::GR, st[(it + 1) & 1]);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      gsync();
      const float* raw = reinterpret_cast<const float*>(cur);
      float2 v[1][8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int x1 = t + m * G::T8;
        v[0][m] = make_float2(raw[(2 * j) * N1 + x1], raw[(2 * j + 1) * N1 + x1]);
      }
      gsync();
      PadX<G::LD> sx{reinterpret_cast<float2*>(cur) + j * G::LD};
      fft_ct<float2, false, N1, 1, 1>(v, t, sx, tw1, gsync);
#pragma unroll
      for (int m = 0; m < 8; ++m) sx.put(0, t + m * G::T8, v[0][m]);
      gsync();
      const size_t x2 = (size_t)r * Q::RPC + (size_t)u * Q::RU + 2 * j;
      float2* ra = P + x2 * Q::H1;
      float2* rbw = ra + Q::H1;
      // Hermitian split of Z = A + i B: A(k) = (Z(k) + conj Z(-k)) / 2, B(k) = (Z(k) - conj Z(-k)) / (2i)
      for (int k = 2 * t; k < Q::H1; k += 2 * G::T8) {
        float2 a[2], b[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float2 zk = sx.get(0, k + e), zm = cconj(sx.get(0, (N1 - k - e) & (N1 - 1)));
          const float2 sm = cadd(zk, zm), d = csub(zk, zm);
          a[e] = make_float2(0.5f * sm.x, 0.5f * sm.y);
          b[e] = make_float2(0.5f * d.y, -0.5f * d.x);
        }
        *reinterpret_cast<float4*>(ra + k) = make_float4(a[0].x, a[0].y, a[1].x, a[1].y);
        *reinterpret_cast<float4*>(rbw + k) = make_float4(b[0].x, b[0].y, b[1].x, b[1].y);
      }
      if (t == 0) {
        // k1 = N1/2: Z(N1/2) = A + i B with A, B real
        const float2 zn = sx.get(0, Q::H1);
        nq[pl * N2 + x2] = zn.x;
        nq[pl * N2 + x2 + 1] = zn.y;
      }
      gsync();
    }
  }

  // 2. every row spectrum of the plane is written (cluster-scope release / acquire)
  cluster.sync();

  // 3. column phase over this CTA's k1 range
  column_phase<N1, N2, CL, NT, false>(P, r * Q::CPC, smraw, tw2);
}

// Inverse.  nq_mode: 0 = the k1 = N1/2 column is zero; 1 = it is nq_scale (C:nq)_c with nq
// holding the row coefficients of eps_p of the six components of the layer.
template <int N1, int N2, int CL, int NT>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT, MinBlocks<NT>::v)
    k_fft2i_l2(float2* __restrict__ spec, const float* __restrict__ nq, float* __restrict__ out,
               const float2* __restrict__ tw1, const float2* __restrict__ tw2, int nq_mode, float nq_scale,
               float lam, float mu, float scale) {
  typedef Pl<N1, N2, CL, NT> Q;
  typedef typename Q::GR_ G;
  extern __shared__ __align__(16) unsigned char smraw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const size_t pl = blockIdx.y;
  float2* P = spec + pl * (size_t)N2 * Q::H1;

  // 1. inverse column FFTs over this CTA's k1 range, in place
  column_phase<N1, N2, CL, NT, true>(P, r * Q::CPC, smraw, tw2);

  // 2. every column of the plane is transformed
  cluster.sync();

  // 3. rows: group g takes row units g, g + GR, ...: stage the unit's half rows (16-byte
  //    L1-bypassing copies), Hermitian rebuild, inverse complex FFT of A + i B, two real rows
  const int g = threadIdx.x / G::NG, lane = threadIdx.x % G::NG;
  const int j = lane / G::T8, t = lane % G::T8;
  const GroupSync<G::NG> gsync{1 + g};
  const size_t z = pl / 6;
  const int c = (int)(pl % 6);
  unsigned char* st[2] = {smraw + (size_t)(2 * g) * Q::ROW_STAGE, smraw + (size_t)(2 * g + 1) * Q::ROW_STAGE};
  const float2* blk0 = P + (size_t)r * Q::RPC * Q::H1;
  auto issue = [&](int u, unsigned char* dst) {
    const float2* s = blk0 + (size_t)u * Q::RU * Q::H1;
    float2* d = reinterpret_cast<float2*>(dst);
    for (int i = lane; i < Q::RU * Q::H1 / 2; i += G::NG) cp_async_16(d + 2 * i, s + 2 * i);
    cp_async_commit();
  };
  if (g < Q::NRU) issue(g, st[0]);
#pragma unroll 1
  for (int it = 0, u = g; u < Q::NRU; ++it, u += Q::GR) {
    unsigned char* cur = st[it & 1];
    if (u + Q::GR < Q::NRU) {
      issue(u + Q::GR, st[(it + 1) & 1]);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    const size_t x2 = (size_t)r * Q::RPC + (size_t)u * Q::RU + 2 * j;
    float na = 0.f, nb = 0.f;
    if (nq_mode) {
      const float* q0 = nq + z * 6 * N2;
      const float tra = q0[x2] + q0[N2 + x2] + q0[2 * N2 + x2];
      const float trb = q0[x2 + 1] + q0[N2 + x2 + 1] + q0[2 * N2 + x2 + 1];
      na = nq_scale * (2.f * mu * q0[c * N2 + x2] + (c < 3 ? lam * tra : 0.f));
      nb = nq_scale * (2.f * mu * q0[c * N2 + x2 + 1] + (c < 3 ? lam * trb : 0.f));
    }
    gsync();
    const float2* sa = reinterpret_cast<const float2*>(cur) + (2 * j) * Q::H1;
    const float2* sb = sa + Q::H1;
    float2 v[1][8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = t + m * G::T8;
      const int kk = k < Q::H1 ? k : (k > Q::H1 ? N1 - k : 0);
      float2 A = sa[kk], B = sb[kk];
      if (k > Q::H1) {
        A = cconj(A);
        B = cconj(B);
      }
      if (k == Q::H1) {
        A = make_float2(na, 0.f);
        B = make_float2(nb, 0.f);
      }
      v[0][m] = cadd(A, cmuli(B));
    }
    gsync();
    PadX<G::LD> sx{reinterpret_cast<float2*>(cur) + j * G::LD};
    fft_ct<float2, true, N1, 1, 1>(v, t, sx, tw1, gsync);
    float* o = out + (pl * N2 + x2) * N1;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int x1 = t + m * G::T8;
      o[x1] = v[0][m].x * scale;
      o[N1 + x1] = v[0][m].y * scale;
    }
    gsync();
  }
}

template <int N1, int N2, int CL, int NT> bool fused_ok() {
  typedef Pl<N1, N2, CL, NT> Q;
  static int ok = -1;  // per process: one device kind per run
  if (ok < 0) {
    ok = 0;
    if (CL > 8) {  // 16-CTA clusters are beyond the portable size
      cudaFuncSetAttribute(k_fft2f_l2<N1, N2, CL, NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      cudaFuncSetAttribute(k_fft2i_l2<N1, N2, CL, NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    if (cudaFuncSetAttribute(k_fft2f_l2<N1, N2, CL, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Q::SMEM) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_fft2i_l2<N1, N2, CL, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Q::SMEM) ==
            cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(CL, 1, 1);
      cfg.blockDim = dim3(NT, 1, 1);
      cfg.dynamicSmemBytes = Q::SMEM;
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = CL;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      cfg.attrs = &at;
      cfg.numAttrs = 1;
      int a = 0, b = 0;
      if (cudaOccupancyMaxActiveClusters(&a, k_fft2f_l2<N1, N2, CL, NT>, &cfg) == cudaSuccess &&
          cudaOccupancyMaxActiveClusters(&b, k_fft2i_l2<N1, N2, CL, NT>, &cfg) == cudaSuccess && a > 0 && b > 0)
        ok = 1;
    }
    cudaGetLastError();
  }
  return ok == 1;
}

template <int N1, int N2, int CL, int NT>
void fwd_n(const fvim_ctx* c, const float* src, int nplanes, const int* zr) {
  k_fft2f_l2<N1, N2, CL, NT><<<dim3(CL, nplanes), NT, Pl<N1, N2, CL, NT>::SMEM, c->stream>>>(
      src, (float2*)c->spec, (float*)c->nq, (const float2*)c->tw1, (const float2*)c->tw2, zr);
}
template <int N1, int N2, int CL, int NT>
void inv_n(const fvim_ctx* c, float* out, int nplanes, int nq_mode, float nq_scale) {
  const float scale = (float)(1.0 / ((double)N1 * (double)N2));
  k_fft2i_l2<N1, N2, CL, NT><<<dim3(CL, nplanes), NT, Pl<N1, N2, CL, NT>::SMEM, c->stream>>>(
      (float2*)c->spec, (const float*)c->nq, out, (const float2*)c->tw1, (const float2*)c->tw2, nq_mode, nq_scale,
      (float)c->lam, (float)c->mu, scale);
}

// plane sizes, cluster sizes and CTA widths: CTAs of at most 64 rows and 32 columns of a
// 512 x 512 plane, 1024-point dimensions in 16-CTA clusters
#define FVIM_L2_SIZES(X)                                                                        \
  X(128, 128, 2, 256) X(256, 128, 4, 256) X(128, 256, 2, 256) X(256, 256, 4, 256)               \
  X(512, 128, 8, 256) X(128, 512, 2, 256)                                                       \
  X(512, 256, 8, 256) X(256, 512, 4, 256) X(512, 512, 8, 256) X(1024, 512, 16, 256)             \
  X(512, 1024, 8, 256) X(1024, 1024, 16, 256)

}  // namespace

bool fft2_fused_available(const fvim_ctx* c) {
  if (c->prec != FVIM_FP32) return false;
#define AV(A, B, K, W) \
  if (c->n1 == A && c->n2 == B) return fused_ok<A, B, K, W>();
  FVIM_L2_SIZES(AV)
#undef AV
  return false;
}

int launch_fft2_fwd_fused(const fvim_ctx* c, const float* src, const int* zr) {
#define FW(A, B, K, W)                        \
  if (c->n1 == A && c->n2 == B) {             \
    fwd_n<A, B, K, W>(c, src, c->nz * 6, zr); \
    FVIM_CUDA_CHECK_LAUNCH();                 \
    return FVIM_OK;                           \
  }
  FVIM_L2_SIZES(FW)
#undef FW
  return FVIM_ERR_UNSUPPORTED;
}

int launch_fft2_inv_fused(const fvim_ctx* c, float* out, int nq_mode, float nq_scale) {
#define IV(A, B, K, W)                                       \
  if (c->n1 == A && c->n2 == B) {                            \
    inv_n<A, B, K, W>(c, out, c->nz * 6, nq_mode, nq_scale); \
    FVIM_CUDA_CHECK_LAUNCH();                                \
    return FVIM_OK;                                          \
  }
  FVIM_L2_SIZES(IV)
#undef IV
  return FVIM_ERR_UNSUPPORTED;
}
