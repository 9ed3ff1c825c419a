// Whole-plane 2-D real FFTs in one pass: one thread-block cluster of CL = 8 CTAs per
// (layer, component) plane, the plane's row spectra held in the cluster's distributed
// shared memory between the row and the column transforms.
//
// Forward (eps_p plane -> half spectrum, Sec. 3.1 discrete Fourier transform):
//   CTA r loads rows x2 in [r R, (r+1) R) (R = N2 / CL, one contiguous block of the
//   plane), transforms them two real rows per complex FFT, splits the Hermitian pairs and
//   keeps the half rows k1 < N1/2 in its shared memory (the k1 = N1/2 coefficient goes to
//   the side array nq); after a cluster barrier CTA r transforms the columns
//   k1 in [r N1/(2 CL), (r+1) N1/(2 CL)), reading element x2 = t + m R of a column from
//   CTA m's shared memory, and writes the spectrum.
// Inverse (half spectrum -> real plane): the same two phases in reverse order; the
//   column results are stored into the owning CTA's shared memory, then each CTA rebuilds
//   the Hermitian rows and writes its real rows.
//
// Each plane is read once and written once: 8 B per voxel and direction in FP32, instead
// of the 16 B of separate row and column kernels.  Hooke's law is not applied here
// (C:eps_p needs all six components of a voxel); the depth kernel applies it per mode,
// and the inverse applies it to the k1 = N1/2 column.
#include <cooperative_groups.h>

#include "fvim_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int CL = 8;    // CTAs per cluster (portable cluster size)
constexpr int NT = 512;  // threads per CTA

template <int N1, int N2> struct Plan {
  static constexpr int H1 = N1 / 2;
  static constexpr int RPC = N2 / CL;            // real rows per CTA
  static constexpr int PAIRS = RPC / 2;          // complex row FFTs per CTA
  static constexpr int T8R = N1 / 8;             // threads per row FFT
  static constexpr int GR = NT / T8R;            // row FFT groups
  static constexpr int NFR = (PAIRS / GR) >= 2 ? 2 : 1;  // row FFTs per thread and pass
  static constexpr int HALVES = PAIRS / (GR * NFR);      // row passes
  static constexpr int PPH = PAIRS / HALVES;     // pairs per pass
  static constexpr int RPH = 2 * PPH;            // real rows per pass
  static constexpr int LDR = H1 + 8;             // padded row-spectrum stride (complex)
  static constexpr int LDX = N1 + N1 / 8;        // padded row-exchange stride (complex)
  static constexpr int T8C = N2 / 8;             // threads per column FFT
  static constexpr int FC = NT / T8C;            // column slots per pass
  static constexpr int CPC = H1 / CL;            // columns per CTA
  static constexpr int NFC = (CPC / FC) >= 2 ? 2 : 1;  // column FFTs per thread and pass
  static constexpr int KCB = FC * NFC;           // columns per pass
  static constexpr int CBATCH = CPC / KCB;       // column passes
  static constexpr int XROW = GR * NFR * LDX;    // complex entries of the row exchange
  static constexpr int XCOL = KCB * N2;          // complex entries of the column exchange
  static constexpr int XRAW = RPH * N1 / 2;      // complex-sized entries of one raw pass
  static constexpr int XCH = XROW > XCOL ? (XROW > XRAW ? XROW : XRAW) : (XCOL > XRAW ? XCOL : XRAW);
  static constexpr int ROWSPEC = RPC * LDR;
  static constexpr size_t SMEM = (size_t)(ROWSPEC + XCH) * sizeof(float2);
  static_assert(T8C == RPC, "column element m must live in CTA m");
  static_assert(GR * T8R == NT && FC * T8C == NT, "thread split");
  static_assert(PAIRS % (GR * NFR) == 0 && HALVES >= 1 && HALVES <= 2, "row passes");
  static_assert(CPC % KCB == 0 && CBATCH >= 1, "column passes");
  static_assert((size_t)(RPH * N1) * sizeof(float) <= (size_t)(RPH * LDR) * sizeof(float2), "raw staging fits");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// padded rows for the row exchange: transform g of this group at buf[g * LDX + p + p/8]
template <typename V, int LD> struct RowX {
  V* buf;
  __device__ __forceinline__ void put(int g, int p, V x) const { buf[g * LD + p + (p >> 3)] = x; }
  __device__ __forceinline__ V get(int g, int p) const { return buf[g * LD + p + (p >> 3)]; }
};
// interleaved columns for the column exchange: entry p of column f + g FC at buf[p KCB + f + g FC]
template <typename V, int KCB, int FC> struct ColX {
  V* buf;
  int f;
  __device__ __forceinline__ void put(int g, int p, V x) const { buf[p * KCB + f + g * FC] = x; }
  __device__ __forceinline__ V get(int g, int p) const { return buf[p * KCB + f + g * FC]; }
};

template <int N1, int N2>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT, 1)
    k_fft2_fwd_cl(const float* __restrict__ src, float2* __restrict__ spec, float* __restrict__ nq,
                  const float2* __restrict__ tw1, const float2* __restrict__ tw2) {
  typedef Plan<N1, N2> P;
  typedef float2 V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* rows = reinterpret_cast<V*>(smraw);  // [RPC][LDR] half row spectra
  V* xch = rows + P::ROWSPEC;             // exchange / staging
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const size_t pl = blockIdx.y;
  const int tid = threadIdx.x;

  // 1. stage the CTA's rows (contiguous in the plane): pass 0 into the exchange area,
  //    pass 1 (if any) into the row-spectrum rows it will become
  const float* blk = src + (pl * N2 + (size_t)r * P::RPC) * N1;
#pragma unroll
  for (int h = 0; h < P::HALVES; ++h) {
    float* dst = h == 0 ? reinterpret_cast<float*>(xch) : reinterpret_cast<float*>(rows + h * P::RPH * P::LDR);
    const float* s = blk + (size_t)h * P::RPH * N1;
    for (int i = tid; i < P::RPH * N1 / 4; i += NT) cp_async_16(dst + 4 * i, s + 4 * i);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }

  // 2. row FFTs, PPH complex transforms per pass
  const int grp = tid / P::T8R, t = tid % P::T8R;
#pragma unroll
  for (int h = 0; h < P::HALVES; ++h) {
    if (h + 1 < P::HALVES) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const float* raw = h == 0 ? reinterpret_cast<const float*>(xch)
                              : reinterpret_cast<const float*>(rows + h * P::RPH * P::LDR);
    V v[P::NFR][8];
#pragma unroll
    for (int f = 0; f < P::NFR; ++f) {
      const int j = grp * P::NFR + f;  // pair within the pass
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int x1 = t + m * P::T8R;
        v[f][m] = make_float2(raw[(2 * j) * N1 + x1], raw[(2 * j + 1) * N1 + x1]);
      }
    }
    __syncthreads();  // the staging area is free from here on
    RowX<V, P::LDX> sx{xch + grp * P::NFR * P::LDX};
    fft_ct<V, false, N1, P::NFR, 1>(v, t, sx, tw1);
#pragma unroll
    for (int f = 0; f < P::NFR; ++f)
#pragma unroll
      for (int m = 0; m < 8; ++m) sx.put(f, t + m * P::T8R, v[f][m]);
    __syncthreads();
    for (int idx = t; idx < P::NFR * (P::H1 + 1); idx += P::T8R) {
      const int f = idx / (P::H1 + 1), k = idx - f * (P::H1 + 1);
      const int j = grp * P::NFR + f;
      const int ra = h * P::RPH + 2 * j;  // local real row of the pair's first member
      const V zk = sx.get(f, k), zmk = cconj(sx.get(f, (N1 - k) & (N1 - 1)));
      const V s = cadd(zk, zmk), d = csub(zk, zmk);
      const V A = make_float2(0.5f * s.x, 0.5f * s.y);
      const V B = make_float2(0.5f * d.y, -0.5f * d.x);
      if (k < P::H1) {
        rows[ra * P::LDR + k] = A;
        rows[(ra + 1) * P::LDR + k] = B;
      } else {
        const size_t x2 = (size_t)r * P::RPC + ra;
        nq[pl * N2 + x2] = A.x;
        nq[pl * N2 + x2 + 1] = B.x;
      }
    }
    __syncthreads();
  }

  // 3. every row spectrum of the plane is in the cluster
  cluster.sync();

  // 4. column FFTs over the CTA's k1 range; element x2 = t + m RPC is row t of CTA m
  const int fcol = tid % P::FC, tc = tid / P::FC;
  const V* peer[CL];
#pragma unroll
  for (int m = 0; m < CL; ++m) peer[m] = cluster.map_shared_rank(rows, m);
#pragma unroll 1
  for (int b = 0; b < P::CBATCH; ++b) {
    const int kb = r * P::CPC + b * P::KCB;
    V v[P::NFC][8];
#pragma unroll
    for (int g = 0; g < P::NFC; ++g)
#pragma unroll
      for (int m = 0; m < 8; ++m) v[g][m] = peer[m][tc * P::LDR + kb + fcol + g * P::FC];
    ColX<V, P::KCB, P::FC> sc{xch, fcol};
    fft_ct<V, false, N2, P::NFC, 1>(v, tc, sc, tw2);
#pragma unroll
    for (int g = 0; g < P::NFC; ++g)
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const size_t k2 = (size_t)tc + m * P::T8C;
        spec[(pl * N2 + k2) * P::H1 + kb + fcol + g * P::FC] = v[g][m];
      }
  }

  // 5. no CTA leaves while a peer may still read its rows
  cluster.sync();
}

// Inverse.  nq_mode: 0 = the k1 = N1/2 column is zero; 1 = it is nq_scale (C:nq)_c with
// nq holding the row coefficients of eps_p of the six components of the layer.
template <int N1, int N2>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT, 1)
    k_fft2_inv_cl(const float2* __restrict__ spec, const float* __restrict__ nq, float* __restrict__ out,
                  const float2* __restrict__ tw1, const float2* __restrict__ tw2, int nq_mode, float nq_scale,
                  float lam, float mu, float scale) {
  typedef Plan<N1, N2> P;
  typedef float2 V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* rows = reinterpret_cast<V*>(smraw);
  V* xch = rows + P::ROWSPEC;
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const size_t pl = blockIdx.y;
  const int tid = threadIdx.x;

  // 1. inverse column FFTs over the CTA's k1 range; x2 = t + m RPC goes to row t of CTA m
  const int fcol = tid % P::FC, tc = tid / P::FC;
  V* peer[CL];
#pragma unroll
  for (int m = 0; m < CL; ++m) peer[m] = cluster.map_shared_rank(rows, m);
#pragma unroll 1
  for (int b = 0; b < P::CBATCH; ++b) {
    const int kb = r * P::CPC + b * P::KCB;
    V v[P::NFC][8];
#pragma unroll
    for (int g = 0; g < P::NFC; ++g)
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const size_t k2 = (size_t)tc + m * P::T8C;
        v[g][m] = spec[(pl * N2 + k2) * P::H1 + kb + fcol + g * P::FC];
      }
    ColX<V, P::KCB, P::FC> sc{xch, fcol};
    fft_ct<V, true, N2, P::NFC, 1>(v, tc, sc, tw2);
#pragma unroll
    for (int g = 0; g < P::NFC; ++g)
#pragma unroll
      for (int m = 0; m < 8; ++m) peer[m][tc * P::LDR + kb + fcol + g * P::FC] = v[g][m];
  }

  // 2. every column result is in its row's CTA
  cluster.sync();

  // 3. Hermitian rows -> two real rows per complex inverse FFT
  const int grp = tid / P::T8R, t = tid % P::T8R;
  const size_t z = pl / 6;
  const int c = (int)(pl % 6);
#pragma unroll 1
  for (int h = 0; h < P::HALVES; ++h) {
    V v[P::NFR][8];
#pragma unroll
    for (int f = 0; f < P::NFR; ++f) {
      const int ra = h * P::RPH + 2 * (grp * P::NFR + f);
      const size_t x2 = (size_t)r * P::RPC + ra;
      float na = 0.f, nb = 0.f;
      if (nq_mode) {
        const float* q0 = nq + z * 6 * N2;
        const float tra = q0[x2] + q0[N2 + x2] + q0[2 * N2 + x2];
        const float trb = q0[x2 + 1] + q0[N2 + x2 + 1] + q0[2 * N2 + x2 + 1];
        na = 2.f * mu * q0[c * N2 + x2] + (c < 3 ? lam * tra : 0.f);
        nb = 2.f * mu * q0[c * N2 + x2 + 1] + (c < 3 ? lam * trb : 0.f);
        na *= nq_scale;
        nb *= nq_scale;
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int k = t + m * P::T8R;
        const int kk = k < P::H1 ? k : (k > P::H1 ? N1 - k : 0);
        V A = rows[ra * P::LDR + kk], B = rows[(ra + 1) * P::LDR + kk];
        if (k > P::H1) {
          A = cconj(A);
          B = cconj(B);
        }
        if (k == P::H1) {
          A = make_float2(na, 0.f);
          B = make_float2(nb, 0.f);
        }
        v[f][m] = cadd(A, cmuli(B));
      }
    }
    RowX<V, P::LDX> sx{xch + grp * P::NFR * P::LDX};
    fft_ct<V, true, N1, P::NFR, 1>(v, t, sx, tw1);
#pragma unroll
    for (int f = 0; f < P::NFR; ++f) {
      const int ra = h * P::RPH + 2 * (grp * P::NFR + f);
      float* o = out + (pl * N2 + (size_t)r * P::RPC + ra) * N1;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int x1 = t + m * P::T8R;
        o[x1] = v[f][m].x * scale;
        o[N1 + x1] = v[f][m].y * scale;
      }
    }
    __syncthreads();  // the exchange area is reused by the next pass
  }
}

template <int N1, int N2> bool cluster_ok() {
  typedef Plan<N1, N2> P;
  static int ok = -1;  // per process: one device kind per run
  if (ok < 0) {
    ok = 0;
    if (cudaFuncSetAttribute(k_fft2_fwd_cl<N1, N2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_fft2_inv_cl<N1, N2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM) ==
            cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(CL, 1, 1);
      cfg.blockDim = dim3(NT, 1, 1);
      cfg.dynamicSmemBytes = P::SMEM;
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = CL;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      cfg.attrs = &at;
      cfg.numAttrs = 1;
      int n1 = 0, n2 = 0;
      if (cudaOccupancyMaxActiveClusters(&n1, k_fft2_fwd_cl<N1, N2>, &cfg) == cudaSuccess &&
          cudaOccupancyMaxActiveClusters(&n2, k_fft2_inv_cl<N1, N2>, &cfg) == cudaSuccess && n1 > 0 && n2 > 0)
        ok = 1;
    }
    cudaGetLastError();
  }
  return ok == 1;
}

template <int N1, int N2> void fwd_n(const fvim_ctx* c, const float* src, int nplanes) {
  k_fft2_fwd_cl<N1, N2><<<dim3(CL, nplanes), NT, Plan<N1, N2>::SMEM, c->stream>>>(
      src, (float2*)c->spec, (float*)c->nq, (const float2*)c->tw1, (const float2*)c->tw2);
}
template <int N1, int N2> void inv_n(const fvim_ctx* c, float* out, int nplanes, int nq_mode, float nq_scale) {
  const float scale = (float)(1.0 / ((double)N1 * (double)N2));
  k_fft2_inv_cl<N1, N2><<<dim3(CL, nplanes), NT, Plan<N1, N2>::SMEM, c->stream>>>(
      (const float2*)c->spec, (const float*)c->nq, out, (const float2*)c->tw1, (const float2*)c->tw2, nq_mode,
      nq_scale, (float)c->lam, (float)c->mu, scale);
}

#define FVIM_CL_SIZES(X) X(256, 256) X(512, 512) X(256, 512) X(512, 256)

}  // namespace

bool fft2_cluster_available(const fvim_ctx* c) {
  if (c->prec != FVIM_FP32) return false;
#define AV(A, B) \
  if (c->n1 == A && c->n2 == B) return cluster_ok<A, B>();
  FVIM_CL_SIZES(AV)
#undef AV
  return false;
}

int launch_fft2_fwd_cluster(const fvim_ctx* c, const float* src) {
#define FW(A, B)                           \
  if (c->n1 == A && c->n2 == B) {          \
    fwd_n<A, B>(c, src, c->nz * 6);        \
    FVIM_CUDA_CHECK_LAUNCH();              \
    return FVIM_OK;                        \
  }
  FVIM_CL_SIZES(FW)
#undef FW
  return FVIM_ERR_UNSUPPORTED;
}

int launch_fft2_inv_cluster(const fvim_ctx* c, float* out, int nq_mode, float nq_scale) {
#define IV(A, B)                                   \
  if (c->n1 == A && c->n2 == B) {                  \
    inv_n<A, B>(c, out, c->nz * 6, nq_mode, nq_scale); \
    FVIM_CUDA_CHECK_LAUNCH();                      \
    return FVIM_OK;                                \
  }
  FVIM_CL_SIZES(IV)
#undef IV
  return FVIM_ERR_UNSUPPORTED;
}
