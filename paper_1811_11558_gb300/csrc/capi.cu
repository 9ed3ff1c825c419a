// C ABI of libfvim (declarations and argument contracts in include/fvim.h).
#include <math.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <utility>
#include <vector>

#include <cudaTypedefs.h>

#include "fvim_internal.cuh"

static thread_local cudaError_t g_last_cuda = cudaSuccess;
static thread_local char g_last_cuda_msg[256];

bool fvim_cuda_failed(cudaError_t e, const char* file, int line) {
  if (e == cudaSuccess) return false;
  g_last_cuda = e;
  const char* base = file ? strrchr(file, '/') : nullptr;
  base = base ? base + 1 : (file ? file : "?");
  snprintf(g_last_cuda_msg, sizeof g_last_cuda_msg, "%s (%s:%d)", cudaGetErrorString(e), base, line);
  return true;
}

namespace {

// J2 radial return with linear isotropic hardening (Sec. 4.1), one thread per voxel.
template <typename T>
__global__ void k_return_map(const T* __restrict__ d_eps, const T* __restrict__ sig_n, const T* __restrict__ ep,
                             T* __restrict__ d_eps_p, T* __restrict__ d_ep, size_t nxy, size_t nvox, T lam, T mu,
                             T sy, T Eh, int* __restrict__ zr) {
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  const size_t z = v / nxy, xy = v - z * nxy;
  const size_t base = z * 6 * nxy + xy;
  T de[6], sg[6], dp[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    de[c] = d_eps[base + c * nxy];
    sg[c] = sig_n[base + c * nxy];
  }
  const T dEp = rmap_voxel(de, sg, ep[v], lam, mu, sy, Eh, dp);
#pragma unroll
  for (int c = 0; c < 6; ++c) d_eps_p[base + c * nxy] = dp[c];
  if (d_ep) d_ep[v] = dEp;
  if (zr && dEp > 0) flow_range_note(zr, (int)z);
}

// S_{n+1} = S_n + increment (Sec. 4.2, update(S)).
template <typename T>
__global__ void k_commit(const T* __restrict__ d_eps, const T* __restrict__ d_eps_p, const T* __restrict__ d_ep,
                         T* __restrict__ sig, T* __restrict__ eps_p, T* __restrict__ ep, size_t nxy, size_t nvox,
                         T lam, T mu) {
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  const size_t z = v / nxy, xy = v - z * nxy;
  const size_t base = z * 6 * nxy + xy;
  T ee[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const T dp = d_eps_p[base + c * nxy];
    ee[c] = d_eps[base + c * nxy] - dp;
    eps_p[base + c * nxy] += dp;
  }
  const T tr = ee[0] + ee[1] + ee[2];
#pragma unroll
  for (int c = 0; c < 6; ++c) sig[base + c * nxy] += 2 * mu * ee[c] + (c < 3 ? lam * tr : (T)0);
  if (d_ep) ep[v] += d_ep[v];
}

struct ProfState {
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[PROF_NSLOTS];
};

const char* kProfNames[PROF_NSLOTS] = {"rows_fwd6", "cols_fwd", "mindlin_depth", "cols_inv", "rows_inv6",
                                       "rows_fwd1", "rows_inv1", "boussinesq", "return_map", "commit",
                                       "fft2_fwd", "fft2_inv"};

// run one launcher, bracketed by events when profiling is on
template <typename F> int timed(fvim_ctx* c, int slot, int& nk, F&& launch) {
  ProfState* ps = (ProfState*)c->prof;
  cudaEvent_t a = nullptr, b = nullptr;
  if (ps && ps->on) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, c->stream);
  }
  const int rc = launch();
  if (a) {
    cudaEventRecord(b, c->stream);
    ps->ev[slot].push_back({a, b});
  }
  if (rc == FVIM_OK) ++nk;
  return rc;
}

size_t elem_size(const fvim_ctx* c) { return c->prec == FVIM_FP64 ? 8 : 4; }
size_t nvox(const fvim_ctx* c) { return (size_t)c->nz * c->n2 * c->n1; }

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

void free_all(fvim_ctx* c) {
  void* bufs[] = {c->z_dev, c->tw1, c->tw2, c->spec, c->nq, c->surf, c->surf_nq, c->st_eps_p, c->st_ep, c->st_sig, c->st_T,
                  c->dev_status};
  for (void* b : bufs)
    if (b) cudaFree(b);
  free(c->z_host);
  free(c->tmap);
  c->tmap = nullptr;
  for (int i = 0; i < FVIM_NSOLVER_BUFS; ++i)
    if (c->sv[i]) { cudaFree(c->sv[i]); c->sv[i] = nullptr; }
  solver_release(c);
  ProfState* ps = (ProfState*)c->prof;
  if (ps) {
    for (auto& v : ps->ev)
      for (auto& e : v) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    delete ps;
    c->prof = nullptr;
  }
}

template <typename T> int upload_twiddles(void** dst, int n) {
  typedef typename Cx<T>::t V;
  std::vector<V> h(n);
  for (int k = 0; k < n; ++k) {
    const double a = -6.283185307179586476925 * (double)k / (double)n;
    h[k] = mk<V>((T)cos(a), (T)sin(a));
  }
  if (FVIM_CU(cudaMalloc(dst, n * sizeof(V)))) return FVIM_ERR_OOM;
  if (FVIM_CU(cudaMemcpy(*dst, h.data(), n * sizeof(V), cudaMemcpyHostToDevice))) return FVIM_ERR_CUDA;
  return FVIM_OK;
}

template <typename T> int upload_nodes(fvim_ctx* c) {
  std::vector<T> h(c->nz);
  for (int i = 0; i < c->nz; ++i) h[i] = (T)c->z_host[i];
  if (FVIM_CU(cudaMalloc(&c->z_dev, c->nz * sizeof(T)))) return FVIM_ERR_OOM;
  if (FVIM_CU(cudaMemcpy(c->z_dev, h.data(), c->nz * sizeof(T), cudaMemcpyHostToDevice))) return FVIM_ERR_CUDA;
  return FVIM_OK;
}

// the driver's tensor-map encoder, looked up once through the runtime (no driver library link)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 f = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return f;
}

// Tensor map of the FP32 depth tile: the spectrum [Nz 6][N2][N1/2] complex seen as a 3-D float
// tensor (2 h1, N2, 6 Nz) with a box of 32 floats (16 complex columns, one 128-byte row) x one
// k2 x B rows, B the largest divisor of 6 Nz up to 256.  FVIM_DEPTH_TMA=0 keeps cp.async.
void setup_depth_tma(fvim_ctx* c) {
  const char* e = getenv("FVIM_DEPTH_TMA");
  if ((e && e[0] == '0') || c->prec != FVIM_FP32 || c->gen || c->h1 < 16) return;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return;
  const int rows = c->nz * 6;
  int box_rows = rows < 256 ? rows : 256;
  while (rows % box_rows) --box_rows;
  void* m = aligned_alloc(64, sizeof(CUtensorMap));
  if (!m) return;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * c->h1, (cuuint64_t)c->n2, (cuuint64_t)rows};
  const cuuint64_t strides[2] = {(cuuint64_t)c->h1 * 8, (cuuint64_t)c->n2 * c->h1 * 8};
  const cuuint32_t box[3] = {32, 1, (cuuint32_t)box_rows};
  const cuuint32_t elem[3] = {1, 1, 1};
  if (enc(reinterpret_cast<CUtensorMap*>(m), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->spec, dims, strides, box, elem,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    free(m);
    return;
  }
  c->tmap = m;
  c->tma_rows = box_rows;
  // test of the expired-wait path: the tile's copies complete, but the mbarrier expects more
  // bytes than they carry, so its phase never completes and the bounded wait runs out
  const char* x = getenv("FVIM_TEST_TMA_EXTRA");
  c->tma_test_extra = x ? atoi(x) : 0;
  if (c->tma_test_extra < 0 || c->tma_test_extra > 4096 || c->tma_test_extra % 16) c->tma_test_extra = 0;
}

}  // namespace

// whole-plane cluster FFTs (FP32, planes that fit a cluster's shared memory), selected by
// the environment variable FVIM_FFT2_CLUSTER=1; the default is the separate row and column
// kernels, which are faster on the 512 x 512 planes measured so far (one cluster of eight
// 209 KB CTAs per plane leaves the load, transform and store phases of a CTA serialised)
static bool use_fft2_cluster(fvim_ctx* c) {
  if (c->fft_path >= 0) return c->fft_path == FVIM_FFT_CLUSTER;
  if (c->fft2_cl < 0) {
    const char* e = getenv("FVIM_FFT2_CLUSTER");
    c->fft2_cl = (e && e[0] == '1' && fft2_cluster_available(c)) ? 1 : 0;
  }
  return c->fft2_cl == 1;
}

// one-pass 2-D FFTs through L2 (FP32 grids of fft2d_l2.cu), selected by the environment
// variable FVIM_FFT2_FUSED=1 (decided once per context); the default is the separate row and
// column kernels, which are faster at 512 x 512 although they move twice the bytes (the
// one-pass kernels are bound by L1 and shared-memory traffic at 24 warps per SM)
static bool use_fft2_fused(fvim_ctx* c) {
  if (c->fft_path >= 0) return c->fft_path == FVIM_FFT_L2;
  if (c->fft2_fused < 0) {
    const char* e = getenv("FVIM_FFT2_FUSED");
    c->fft2_fused = (e && e[0] == '1' && fft2_fused_available(c)) ? 1 : 0;
  }
  return c->fft2_fused == 1;
}

bool fft_path_available(const fvim_ctx* c, int path) {
  if (path == FVIM_FFT_ROWCOL) return true;
  if (c->gen || c->prec != FVIM_FP32) return false;
  if (path == FVIM_FFT_L2) return fft2_fused_available(c);
  if (path == FVIM_FFT_CLUSTER) return fft2_cluster_available(c);
  return false;
}

// Mindlin apply in three passes: 2-D FFT of the eps_p planes, the depth operator with Hooke's
// law per mode, inverse 2-D FFT (the k1 = N1/2 column of the stress output is -C:eps_p, times
// N2 because it skips the column transforms that the 1/(N1 N2) normalisation undoes)
template <typename T> int apply_mindlin_fused(fvim_ctx* c, const T* eps_p, T* out, int kind, T* u3, const int* zr,
                                              int& nk) {
  if constexpr (sizeof(T) == 4) {
    int rc;
    if ((rc = timed(c, PROF_FFT2_FWD, nk, [&] { return launch_fft2_fwd_fused(c, eps_p, zr); }))) return rc;
    if ((rc = timed(c, PROF_MINDLIN_DEPTH, nk,
                    [&] { return launch_mindlin_depth<T>(c, kind, u3 != nullptr, true, zr); })))
      return rc;
    const int mode = kind == FVIM_STRESS ? 1 : 0;
    if ((rc = timed(c, PROF_FFT2_INV, nk, [&] { return launch_fft2_inv_fused(c, out, mode, -(float)c->n2); })))
      return rc;
    return FVIM_OK;
  } else {
    return FVIM_ERR_UNSUPPORTED;
  }
}

template <typename T> int apply_mindlin_cluster(fvim_ctx* c, const T* eps_p, T* out, int kind, T* u3, int& nk) {
  if constexpr (sizeof(T) == 4) {
    int rc;
    if ((rc = timed(c, PROF_FFT2_FWD, nk, [&] { return launch_fft2_fwd_cluster(c, eps_p); }))) return rc;
    if ((rc = timed(c, PROF_MINDLIN_DEPTH, nk, [&] { return launch_mindlin_depth<T>(c, kind, u3 != nullptr, true); })))
      return rc;
    // stress output: the k1 = N1/2 column (no operator term) is -C:eps_p, times N2 because
    // it skips the column transforms that the 1/(N1 N2) normalisation undoes
    const int mode = kind == FVIM_STRESS ? 1 : 0;
    if ((rc = timed(c, PROF_FFT2_INV, nk, [&] { return launch_fft2_inv_cluster(c, out, mode, -(float)c->n2); })))
      return rc;
    return FVIM_OK;
  } else {
    return FVIM_ERR_UNSUPPORTED;
  }
}

// Mindlin apply on a direct-DFT grid: row and column DFTs of the eps_p planes, the depth
// operator with Hooke's law per mode (Nyquist modes of even sides and the padding columns
// carry no operator term there), column and row inverse DFTs; the surface displacement
// spectrum takes the same inverse path
template <typename T> int apply_mindlin_gen(fvim_ctx* c, const T* eps_p, T* out, int kind, T* u3, int& nk) {
  int rc;
  const size_t planes = (size_t)c->nz * 6;
  const T scale = (T)(1.0 / ((double)c->n1 * (double)c->n2));
  if ((rc = timed(c, PROF_ROWS_FWD6, nk, [&] { return launch_dft_rows_fwd<T>(c, eps_p, c->spec, planes * c->n2); })))
    return rc;
  if ((rc = timed(c, PROF_COLS_FWD, nk, [&] { return launch_dft_cols<T>(c, false, c->spec, (int)planes); }))) return rc;
  if ((rc = timed(c, PROF_MINDLIN_DEPTH, nk, [&] { return launch_mindlin_depth<T>(c, kind, u3 != nullptr, true); })))
    return rc;
  if ((rc = timed(c, PROF_COLS_INV, nk, [&] { return launch_dft_cols<T>(c, true, c->spec, (int)planes); }))) return rc;
  if ((rc = timed(c, PROF_ROWS_INV6, nk,
                  [&] { return launch_dft_rows_inv<T>(c, c->spec, out, planes * c->n2, scale); })))
    return rc;
  if (u3) {
    if ((rc = timed(c, PROF_COLS_INV, nk, [&] { return launch_dft_cols<T>(c, true, c->surf, 1); }))) return rc;
    if ((rc = timed(c, PROF_ROWS_INV1, nk, [&] { return launch_dft_rows_inv<T>(c, c->surf, u3, c->n2, scale); })))
      return rc;
  }
  return FVIM_OK;
}

// Boussinesq apply on a direct-DFT grid (same sequence as the FFT path, direct DFTs)
template <typename T> int apply_boussinesq_gen(fvim_ctx* c, const T* p, T* u3, T* vol, int kind, int& nk) {
  int rc;
  const T scale = (T)(1.0 / ((double)c->n1 * (double)c->n2));
  if ((rc = timed(c, PROF_ROWS_FWD1, nk, [&] { return launch_dft_rows_fwd<T>(c, p, c->surf, c->n2); }))) return rc;
  if ((rc = timed(c, PROF_COLS_FWD, nk, [&] { return launch_dft_cols<T>(c, false, c->surf, 1); }))) return rc;
  if ((rc = timed(c, PROF_BOUSSINESQ, nk,
                  [&] { return launch_boussinesq<T>(c, kind, vol != nullptr, u3 != nullptr); })))
    return rc;
  if (vol) {
    const size_t planes = (size_t)c->nz * 6;
    if ((rc = timed(c, PROF_COLS_INV, nk, [&] { return launch_dft_cols<T>(c, true, c->spec, (int)planes); })))
      return rc;
    if ((rc = timed(c, PROF_ROWS_INV6, nk,
                    [&] { return launch_dft_rows_inv<T>(c, c->spec, vol, planes * c->n2, scale); })))
      return rc;
  }
  if (u3) {
    if ((rc = timed(c, PROF_COLS_INV, nk, [&] { return launch_dft_cols<T>(c, true, c->surf, 1); }))) return rc;
    if ((rc = timed(c, PROF_ROWS_INV1, nk, [&] { return launch_dft_rows_inv<T>(c, c->surf, u3, c->n2, scale); })))
      return rc;
  }
  return FVIM_OK;
}

template <typename T> int apply_mindlin_t(fvim_ctx* c, const T* eps_p, T* out, int kind, T* u3, const int* zr) {
  int rc;
  int nk = 0;
  if (c->gen) {
    if ((rc = apply_mindlin_gen<T>(c, eps_p, out, kind, u3, nk))) return rc;
    c->last_kernels = nk;
    return FVIM_OK;
  }
  if (use_fft2_cluster(c)) {
    if ((rc = apply_mindlin_cluster<T>(c, eps_p, out, kind, u3, nk))) return rc;
    if (u3) {
      if ((rc = timed(c, PROF_COLS_INV, nk, [&] { return launch_cols<T>(c, true, c->surf, 1); }))) return rc;
      if ((rc = timed(c, PROF_ROWS_INV1, nk, [&] { return launch_rows_inv1<T>(c, u3); }))) return rc;
    }
    c->last_kernels = nk;
    return FVIM_OK;
  }
  // a known layer range of the input skips the forward passes of the empty layers (the
  // Nyquist side array of those layers is left stale, so only for strain output)
  const int* zin = kind == FVIM_STRAIN ? zr : nullptr;
  if (sizeof(T) == 4 && use_fft2_fused(c)) {
    if ((rc = apply_mindlin_fused<T>(c, eps_p, out, kind, u3, zin, nk))) return rc;
    if (u3) {
      if ((rc = timed(c, PROF_COLS_INV, nk, [&] { return launch_cols<T>(c, true, c->surf, 1); }))) return rc;
      if ((rc = timed(c, PROF_ROWS_INV1, nk, [&] { return launch_rows_inv1<T>(c, u3); }))) return rc;
    }
    c->last_kernels = nk;
    return FVIM_OK;
  }
  if ((rc = timed(c, PROF_ROWS_FWD6, nk, [&] { return launch_rows_fwd6<T>(c, eps_p, 0, c->nz, zin); }))) return rc;
  if ((rc = timed(c, PROF_COLS_FWD, nk, [&] { return launch_cols<T>(c, false, c->spec, c->nz * 6, zin); })))
    return rc;
  if ((rc = timed(c, PROF_MINDLIN_DEPTH, nk,
                  [&] { return launch_mindlin_depth<T>(c, kind, u3 != nullptr, false, zin); })))
    return rc;
  if ((rc = timed(c, PROF_COLS_INV, nk, [&] { return launch_cols<T>(c, true, c->spec, c->nz * 6); }))) return rc;
  if ((rc = timed(c, PROF_ROWS_INV6, nk, [&] {
         // the k1 = N1/2 column never goes through the column transforms, so it carries
         // the factor N2 that the 1/(N1 N2) normalisation of rows_inv6 removes
         return launch_rows_inv6<T>(c, out, kind == FVIM_STRESS ? -(T)c->n2 : (T)0, 0, c->nz);
       })))
    return rc;
  if (u3) {
    if ((rc = timed(c, PROF_COLS_INV, nk, [&] { return launch_cols<T>(c, true, c->surf, 1); }))) return rc;
    if ((rc = timed(c, PROF_ROWS_INV1, nk, [&] { return launch_rows_inv1<T>(c, u3); }))) return rc;
  }
  c->last_kernels = nk;
  return FVIM_OK;
}

template <typename T> int apply_boussinesq_t(fvim_ctx* c, const T* p, T* u3, T* vol, int kind) {
  int rc;
  int nk = 0;
  if (c->gen) {
    if ((rc = apply_boussinesq_gen<T>(c, p, u3, vol, kind, nk))) return rc;
    c->last_kernels = nk;
    return FVIM_OK;
  }
  if (u3 && !vol && c->n2 >= 16) {
    // surface displacement only: rows, fused column pass (transform, compliance, inverse), rows
    bool fused = false;
    if ((rc = timed(c, PROF_ROWS_FWD1, nk, [&] { return launch_rows_fwd1<T>(c, p); }))) return rc;
    if ((rc = timed(c, PROF_BOUSSINESQ, nk, [&] {
           fused = launch_cols_conv_ct<T>(c);
           FVIM_CUDA_CHECK_LAUNCH();
           return FVIM_OK;
         })))
      return rc;
    if (fused) {
      if ((rc = timed(c, PROF_ROWS_INV1, nk, [&] { return launch_rows_inv1<T>(c, u3); }))) return rc;
      c->last_kernels = nk;
      return FVIM_OK;
    }
    nk = 0;  // no variant for this N2: the general sequence below
  }
  if ((rc = timed(c, PROF_ROWS_FWD1, nk, [&] { return launch_rows_fwd1<T>(c, p); }))) return rc;
  if ((rc = timed(c, PROF_COLS_FWD, nk, [&] { return launch_cols<T>(c, false, c->surf, 1); }))) return rc;
  if ((rc = timed(c, PROF_BOUSSINESQ, nk,
                  [&] { return launch_boussinesq<T>(c, kind, vol != nullptr, u3 != nullptr); })))
    return rc;
  if (vol && sizeof(T) == 4 && use_fft2_fused(c)) {
    if ((rc = timed(c, PROF_FFT2_INV, nk, [&] { return launch_fft2_inv_fused(c, (float*)vol, 0, 0.f); }))) return rc;
  } else if (vol && sizeof(T) == 4 && use_fft2_cluster(c)) {
    if ((rc = timed(c, PROF_FFT2_INV, nk, [&] { return launch_fft2_inv_cluster(c, (float*)vol, 0, 0.f); }))) return rc;
  } else if (vol) {
    if ((rc = timed(c, PROF_COLS_INV, nk, [&] { return launch_cols<T>(c, true, c->spec, c->nz * 6); }))) return rc;
    if ((rc = timed(c, PROF_ROWS_INV6, nk, [&] { return launch_rows_inv6<T>(c, vol, (T)0, 0, c->nz); }))) return rc;
  }
  if (u3) {
    if ((rc = timed(c, PROF_COLS_INV, nk, [&] { return launch_cols<T>(c, true, c->surf, 1); }))) return rc;
    if ((rc = timed(c, PROF_ROWS_INV1, nk, [&] { return launch_rows_inv1<T>(c, u3); }))) return rc;
  }
  c->last_kernels = nk;
  return FVIM_OK;
}

template <typename T>
int return_map_t(fvim_ctx* c, const T* d_eps, T* d_eps_p, T* d_ep, int* zr) {
  const size_t nv = nvox(c);
  const int threads = 256;
  const unsigned blocks = (unsigned)((nv + threads - 1) / threads);
  int nk = 0;
  const int rc = timed(c, PROF_RETURN_MAP, nk, [&] {
    k_return_map<T><<<blocks, threads, 0, c->stream>>>(d_eps, (const T*)c->st_sig, (const T*)c->st_ep, d_eps_p, d_ep,
                                                       (size_t)c->n1 * c->n2, nv, (T)c->lam, (T)c->mu,
                                                       (T)c->sigma_y, (T)c->E_h, zr);
    FVIM_CUDA_CHECK_LAUNCH();
    return FVIM_OK;
  });
  c->last_kernels = nk;
  return rc;
}

template <typename T> int commit_t(fvim_ctx* c, const T* d_eps, const T* d_eps_p, const T* d_ep) {
  const size_t nv = nvox(c);
  const int threads = 256;
  const unsigned blocks = (unsigned)((nv + threads - 1) / threads);
  int nk = 0;
  const int rc = timed(c, PROF_COMMIT, nk, [&] {
    k_commit<T><<<blocks, threads, 0, c->stream>>>(d_eps, d_eps_p, d_ep, (T*)c->st_sig, (T*)c->st_eps_p,
                                                   (T*)c->st_ep, (size_t)c->n1 * c->n2, nv, (T)c->lam, (T)c->mu);
    FVIM_CUDA_CHECK_LAUNCH();
    return FVIM_OK;
  });
  c->last_kernels = nk;
  return rc;
}

template int apply_mindlin_t<float>(fvim_ctx*, const float*, float*, int, float*, const int*);
template int apply_mindlin_t<double>(fvim_ctx*, const double*, double*, int, double*, const int*);
template int apply_boussinesq_t<float>(fvim_ctx*, const float*, float*, float*, int);
template int apply_boussinesq_t<double>(fvim_ctx*, const double*, double*, double*, int);
template int return_map_t<float>(fvim_ctx*, const float*, float*, float*, int*);
template int return_map_t<double>(fvim_ctx*, const double*, double*, double*, int*);
template int commit_t<float>(fvim_ctx*, const float*, const float*, const float*);
template int commit_t<double>(fvim_ctx*, const double*, const double*, const double*);

bool grid_gen(int n1, int n2) { return !is_pow2(n1) || !is_pow2(n2); }

bool grid_ok(int n1, int n2) {
  const bool p1 = is_pow2(n1) && n1 >= 4 && n1 <= 1024, p2 = is_pow2(n2) && n2 >= 2 && n2 <= 1024;
  if (p1 && p2) return true;
  // direct-DFT grids: odd sides 3..255, the other side odd or a power of two up to 256
  const bool o1 = (n1 & 1) && n1 >= 3 && n1 <= 255, o2 = (n2 & 1) && n2 >= 3 && n2 <= 255;
  const bool q1 = is_pow2(n1) && n1 >= 4 && n1 <= 256, q2 = is_pow2(n2) && n2 >= 2 && n2 <= 256;
  return (o1 || q1) && (o2 || q2) && (o1 || o2);
}

int spec_stride(int n1, int n2) { return grid_gen(n1, n2) ? (n1 / 2 + 1 + 15) / 16 * 16 : n1 / 2; }

extern "C" {

const char* fvim_last_cuda_error(void) { return g_last_cuda == cudaSuccess ? "no error" : g_last_cuda_msg; }

const char* fvim_strerror(int s) {
  switch (s) {
    case FVIM_OK: return "ok";
    case FVIM_ERR_ARG: return "invalid argument";
    case FVIM_ERR_OOM: return "device allocation failed";
    case FVIM_ERR_CUDA: return "CUDA error";
    case FVIM_ERR_NONFINITE: return "non-finite value";
    case FVIM_ERR_NOT_CONVERGED: return "not converged";
    case FVIM_ERR_TIMEOUT: return "bounded wait expired";
    case FVIM_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

int fvim_create(fvim_ctx** out, int n1, int n2, int nz, const double* z_nodes, double L1, double L2, int precision,
                void* stream) {
  if (!out) return FVIM_ERR_ARG;
  *out = nullptr;
  if (!grid_ok(n1, n2)) return FVIM_ERR_ARG;
  if (nz < 2 || nz > 512 || !z_nodes) return FVIM_ERR_ARG;
  if (!(L1 > 0) || !(L2 > 0)) return FVIM_ERR_ARG;
  if (precision != FVIM_FP32 && precision != FVIM_FP64) return FVIM_ERR_ARG;
  if (z_nodes[0] != 0.0) return FVIM_ERR_ARG;
  for (int i = 1; i < nz; ++i)
    if (!(z_nodes[i] > z_nodes[i - 1]) || !isfinite(z_nodes[i])) return FVIM_ERR_ARG;
  fvim_ctx* c = new (std::nothrow) fvim_ctx();
  if (!c) return FVIM_ERR_OOM;
  memset(c, 0, sizeof(*c));
  c->fft2_cl = -1;
  c->fft2_fused = -1;
  c->fft_path = -1;
  c->n1 = n1;
  c->n2 = n2;
  c->nz = nz;
  c->gen = grid_gen(n1, n2) ? 1 : 0;
  c->h1 = spec_stride(n1, n2);
  c->hs = c->gen ? n1 / 2 + 1 : c->h1;
  c->prec = precision;
  c->L1 = L1;
  c->L2 = L2;
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  c->z_host = (double*)malloc(nz * sizeof(double));
  if (!c->z_host) { delete c; return FVIM_ERR_OOM; }
  memcpy(c->z_host, z_nodes, nz * sizeof(double));
  const double h = z_nodes[1] - z_nodes[0];
  c->uniform = 1;
  for (int i = 1; i < nz; ++i)
    if (fabs((z_nodes[i] - z_nodes[i - 1]) - h) > 1e-12 * fabs(z_nodes[nz - 1])) c->uniform = 0;
  c->hz = h;
  fvim_set_material(c, 1.0, 0.3, INFINITY, 0.0);
  // a grid tuned earlier in this process starts with its tuned tile plan and FFT path
  if ((c->depth_chunk = plan_lookup(c)) > 0) c->plan_tuned = 1;
  c->fft_path = plan_lookup_fft(c);
  c->depth_ctas = plan_lookup_ctas(c);
  c->depth_cut = FVIM_DEPTH_CUTOFF_DEFAULT;
  int rc;
  const size_t es = precision == FVIM_FP64 ? 8 : 4;
  const size_t cs = 2 * es;
  if (precision == FVIM_FP64) {
    if ((rc = upload_twiddles<double>(&c->tw1, n1)) || (rc = upload_twiddles<double>(&c->tw2, n2)) ||
        (rc = upload_nodes<double>(c))) { free_all(c); delete c; return rc; }
  } else {
    if ((rc = upload_twiddles<float>(&c->tw1, n1)) || (rc = upload_twiddles<float>(&c->tw2, n2)) ||
        (rc = upload_nodes<float>(c))) { free_all(c); delete c; return rc; }
  }
  const size_t nv = nvox(c);
  struct { void** p; size_t bytes; } al[] = {
      {&c->spec, (size_t)nz * 6 * n2 * c->h1 * cs}, {&c->nq, (size_t)nz * 6 * n2 * es},
      {&c->surf, (size_t)n2 * c->h1 * cs},          {&c->surf_nq, (size_t)n2 * es},
      {&c->st_eps_p, nv * 6 * es},                   {&c->st_ep, nv * es},
      {&c->st_sig, nv * 6 * es},                   {&c->st_T, (size_t)n2 * n1 * es}};
  for (auto& a : al) {
    if (FVIM_CU(cudaMalloc(a.p, a.bytes))) { cudaGetLastError(); free_all(c); delete c; return FVIM_ERR_OOM; }
    if (FVIM_CU(cudaMemset(*a.p, 0, a.bytes))) { free_all(c); delete c; return FVIM_ERR_CUDA; }
  }
  if (FVIM_CU(cudaMalloc((void**)&c->dev_status, 16))) { cudaGetLastError(); free_all(c); delete c; return FVIM_ERR_OOM; }
  if (FVIM_CU(cudaMemset(c->dev_status, 0, 16))) { free_all(c); delete c; return FVIM_ERR_CUDA; }
  setup_depth_tma(c);
  // the fills above run on the legacy stream; wait for them without touching other streams
  // (another thread may be capturing a graph on its own non-blocking stream)
  if (FVIM_CU(cudaStreamSynchronize(cudaStreamLegacy))) { free_all(c); delete c; return FVIM_ERR_CUDA; }
  *out = c;
  return FVIM_OK;
}

int fvim_set_material(fvim_ctx* c, double E, double nu, double sigma_y, double E_h) {
  if (!c) return FVIM_ERR_ARG;
  if (!(E > 0) || !(nu > -1.0 && nu < 0.5) || !(sigma_y > 0) || !(E_h >= 0)) return FVIM_ERR_ARG;
  // captured solver graphs hold the material constants as kernel arguments
  if (E != c->E || nu != c->nu || sigma_y != c->sigma_y || E_h != c->E_h) solver_drop_graphs(c);
  c->E = E;
  c->nu = nu;
  c->sigma_y = sigma_y;
  c->E_h = E_h;
  c->mu = E / (2.0 * (1.0 + nu));
  c->lam = 2.0 * c->mu * nu / (1.0 - 2.0 * nu);
  return FVIM_OK;
}

int fvim_set_stream(fvim_ctx* c, void* stream) {
  if (!c) return FVIM_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  return FVIM_OK;
}

int fvim_apply_mindlin(fvim_ctx* c, const void* eps_p, void* out, int out_kind, void* u3) {
  if (!c || !eps_p || !out || eps_p == out) return FVIM_ERR_ARG;
  if (out_kind != FVIM_STRESS && out_kind != FVIM_STRAIN) return FVIM_ERR_ARG;
  c->last_kernels = 0;
  if (c->prec == FVIM_FP64) return apply_mindlin_t<double>(c, (const double*)eps_p, (double*)out, out_kind, (double*)u3);
  return apply_mindlin_t<float>(c, (const float*)eps_p, (float*)out, out_kind, (float*)u3);
}

static_assert(FVIM_GROUP_MAX == kGrpMax, "group size of the C ABI and of the kernels");

int fvim_apply_mindlin_group(fvim_ctx* const* ctx, int n, const void* const* eps_p, void* const* out, int out_kind,
                             void* stream) {
  if (!ctx || !eps_p || !out || n < 1 || n > FVIM_GROUP_MAX) return FVIM_ERR_ARG;
  if (out_kind != FVIM_STRESS && out_kind != FVIM_STRAIN) return FVIM_ERR_ARG;
  GrpTable t;
  memset(&t, 0, sizeof(t));
  t.n = n;
  for (int i = 0; i < n; ++i) {
    const fvim_ctx* c = ctx[i];
    if (!c || !eps_p[i] || !out[i] || eps_p[i] == out[i]) return FVIM_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctx[j] == c || out[j] == out[i]) return FVIM_ERR_ARG;
    const bool pow2 = (c->n1 & (c->n1 - 1)) == 0 && (c->n2 & (c->n2 - 1)) == 0;
    if (c->prec != FVIM_FP32 || c->gen || !pow2 || c->n1 < 64 || c->n1 > 512 || c->n2 < 64 || c->n2 > 512 ||
        c->nz < 4 || c->nz > 64)
      return FVIM_ERR_UNSUPPORTED;
    GrpProb& P = t.p[i];
    P.eps = (const float*)eps_p[i];
    P.out = (float*)out[i];
    P.spec = (float2*)c->spec;
    P.nq = (float*)c->nq;
    P.tw1 = (const float2*)c->tw1;
    P.tw2 = (const float2*)c->tw2;
    P.zn = (const float*)c->z_dev;
    P.n1 = c->n1;
    P.n2 = c->n2;
    P.nz = c->nz;
    P.h1 = c->h1;
    P.hs = c->hs;
    P.nch = (c->nz + 3) / 4;
    P.nchp = 1;
    while (P.nchp < P.nch) P.nchp <<= 1;
    P.uniform = c->uniform;
    P.out_kind = out_kind;
    const double two_pi = 6.283185307179586476925;
    P.w1 = (float)(two_pi / c->L1);
    P.w2 = (float)(two_pi / c->L2);
    P.lam = (float)c->lam;
    P.mu = (float)c->mu;
    P.nu = (float)c->nu;
    P.hz = (float)c->hz;
    P.cut = c->depth_cut;
    // the k1 = N1/2 column never goes through the column transforms, so it carries the
    // factor N2 that the 1/(N1 N2) normalisation of the inverse rows removes
    P.nq_scale = out_kind == FVIM_STRESS ? -(float)c->n2 : 0.f;
    P.scale = (float)(1.0 / ((double)c->n1 * (double)c->n2));
  }
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if ((rc = launch_grp_rows_fwd(t, s))) return rc;
  if ((rc = launch_grp_cols(t, false, s))) return rc;
  if ((rc = launch_grp_depth(t, s))) return rc;
  if ((rc = launch_grp_cols(t, true, s))) return rc;
  return launch_grp_rows_inv(t, s);
}

int fvim_apply_boussinesq(fvim_ctx* c, const void* p, void* u3, void* vol, int out_kind) {
  if (!c || !p || (!u3 && !vol)) return FVIM_ERR_ARG;
  if (out_kind != FVIM_STRESS && out_kind != FVIM_STRAIN) return FVIM_ERR_ARG;
  c->last_kernels = 0;
  if (c->prec == FVIM_FP64)
    return apply_boussinesq_t<double>(c, (const double*)p, (double*)u3, (double*)vol, out_kind);
  return apply_boussinesq_t<float>(c, (const float*)p, (float*)u3, (float*)vol, out_kind);
}

int fvim_return_map(fvim_ctx* c, const void* d_eps, void* d_eps_p, void* d_ep) {
  if (!c || !d_eps || !d_eps_p || d_eps == d_eps_p) return FVIM_ERR_ARG;
  if (!isfinite(c->sigma_y)) return FVIM_ERR_ARG;
  if (c->prec == FVIM_FP64) return return_map_t<double>(c, (const double*)d_eps, (double*)d_eps_p, (double*)d_ep);
  return return_map_t<float>(c, (const float*)d_eps, (float*)d_eps_p, (float*)d_ep);
}

int fvim_commit_state(fvim_ctx* c, const void* d_eps, const void* d_eps_p, const void* d_ep) {
  if (!c || !d_eps || !d_eps_p) return FVIM_ERR_ARG;
  if (c->prec == FVIM_FP64)
    return commit_t<double>(c, (const double*)d_eps, (const double*)d_eps_p, (const double*)d_ep);
  return commit_t<float>(c, (const float*)d_eps, (const float*)d_eps_p, (const float*)d_ep);
}

int fvim_get_state(fvim_ctx* c, void* eps_p, void* e_p, void* sigma) {
  if (!c) return FVIM_ERR_ARG;
  const size_t es = elem_size(c), nv = nvox(c);
  if (eps_p && FVIM_CU(cudaMemcpyAsync(eps_p, c->st_eps_p, nv * 6 * es, cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
  if (e_p && FVIM_CU(cudaMemcpyAsync(e_p, c->st_ep, nv * es, cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
  if (sigma && FVIM_CU(cudaMemcpyAsync(sigma, c->st_sig, nv * 6 * es, cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
  return FVIM_OK;
}

int fvim_set_state(fvim_ctx* c, const void* eps_p, const void* e_p, const void* sigma) {
  if (!c) return FVIM_ERR_ARG;
  const size_t es = elem_size(c), nv = nvox(c);
  if (eps_p && FVIM_CU(cudaMemcpyAsync(c->st_eps_p, eps_p, nv * 6 * es, cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
  if (e_p && FVIM_CU(cudaMemcpyAsync(c->st_ep, e_p, nv * es, cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
  if (sigma && FVIM_CU(cudaMemcpyAsync(c->st_sig, sigma, nv * 6 * es, cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
  return FVIM_OK;
}

int fvim_reset_state(fvim_ctx* c) {
  if (!c) return FVIM_ERR_ARG;
  const size_t es = elem_size(c), nv = nvox(c);
  if (FVIM_CU(cudaMemsetAsync(c->st_eps_p, 0, nv * 6 * es, c->stream)) ||
      FVIM_CU(cudaMemsetAsync(c->st_ep, 0, nv * es, c->stream)) ||
      FVIM_CU(cudaMemsetAsync(c->st_sig, 0, nv * 6 * es, c->stream)) ||
      FVIM_CU(cudaMemsetAsync(c->st_T, 0, (size_t)c->n1 * c->n2 * es, c->stream)))
    return FVIM_ERR_CUDA;
  return FVIM_OK;
}

size_t fvim_footprint(int n1, int n2, int nz, int precision) {
  if (n1 < 1 || n2 < 1 || nz < 1) return 0;
  const size_t es = precision == FVIM_FP64 ? 8 : 4;
  const size_t ns = (size_t)n1 * n2, nv = ns * nz;
  const size_t h = (size_t)spec_stride(n1, n2);
  const size_t spec = (size_t)nz * 6 * n2 * h * 2 * es + (size_t)nz * 6 * n2 * es;
  const size_t state = nv * 6 * es * 2 + nv * es + ns * es;
  const size_t solver = 8 * nv * 6 * es + nv * es + 13 * ns * es + 64 * 1024;
  return spec + state + solver + (size_t)(n1 + n2) * 2 * es + (size_t)n2 * h * 2 * es;
}

int fvim_sync(fvim_ctx* c) {
  if (!c) return FVIM_ERR_ARG;
  if (FVIM_CU(cudaStreamSynchronize(c->stream))) return FVIM_ERR_CUDA;
  if (c->dev_status) {
    int st = 0;
    if (FVIM_CU(cudaMemcpyAsync(&st, c->dev_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) ||
        FVIM_CU(cudaStreamSynchronize(c->stream)))
      return FVIM_ERR_CUDA;
    if (st) {
      if (FVIM_CU(cudaMemsetAsync(c->dev_status, 0, sizeof(int), c->stream))) return FVIM_ERR_CUDA;
      return FVIM_ERR_TIMEOUT;
    }
  }
  return FVIM_OK;
}

int fvim_destroy(fvim_ctx* c) {
  if (!c) return FVIM_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  return FVIM_OK;
}

int fvim_last_kernel_count(const fvim_ctx* c) { return c ? c->last_kernels : 0; }

int fvim_profile_enable(fvim_ctx* c, int on) {
  if (!c) return FVIM_ERR_ARG;
  if (!c->prof) {
    c->prof = new (std::nothrow) ProfState();
    if (!c->prof) return FVIM_ERR_OOM;
  }
  ((ProfState*)c->prof)->on = on != 0;
  return FVIM_OK;
}

int fvim_profile_read(fvim_ctx* c, double* total_ms, int* launches, int nslots) {
  if (!c || nslots < 0 || (nslots && (!total_ms || !launches))) return FVIM_ERR_ARG;
  for (int s = 0; s < nslots; ++s) { total_ms[s] = 0; launches[s] = 0; }
  ProfState* ps = (ProfState*)c->prof;
  if (!ps) return FVIM_OK;
  if (FVIM_CU(cudaStreamSynchronize(c->stream))) return FVIM_ERR_CUDA;
  for (int s = 0; s < PROF_NSLOTS; ++s) {
    for (auto& e : ps->ev[s]) {
      float ms = 0;
      cudaEventElapsedTime(&ms, e.first, e.second);
      if (s < nslots) { total_ms[s] += ms; launches[s] += 1; }
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    ps->ev[s].clear();
  }
  return FVIM_OK;
}

const char* fvim_profile_name(int slot) { return (slot >= 0 && slot < PROF_NSLOTS) ? kProfNames[slot] : nullptr; }

}  // extern "C"
