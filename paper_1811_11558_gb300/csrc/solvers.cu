// Solvers of the elastic-plastic contact problem (declarations in include/fvim.h):
//   * elastic contact: constrained conjugate gradient of Polonsky & Keer (1999) on the dual
//     problem with the total-load constraint (Sec. 5.1, Eq. total_pressure);
//   * plastic increment: DF-SANE of La Cruz, Martinez & Raydan (2006) on the residual of
//     the implicit incremental equation (Sec. 4.2, Sec. 4.3);
//   * coupling: Algorithm 1 (Sec. 5.2).
// Vectors stay on the device in the context's precision.  Every reduction is a grid of
// fixed blocks writing FP64 partial sums that the last block to finish adds in block order
// (the host-loop fallbacks add them on the host in the same order), so results are bitwise
// reproducible.  The CG's scalar logic runs in single-block finisher kernels; the CG
// iterations and DF-SANE's iterations with its line search each run as a device-side loop (a
// WHILE node of one captured graph) whose state the host reads once per solve (batches of
// captured CG iterations with one status read each as the fallback).  Every loop is capped.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "fvim_internal.cuh"

namespace {

constexpr int RT = 256;       // threads of a reduction block
constexpr int RMAXB = 1024;   // blocks of a reduction grid
constexpr int NVMAX = 3;      // values reduced per pass
constexpr size_t kScalarBlock = 256;  // bytes of the solver's device scalar block (V_PKS)
constexpr size_t kDfsBytes = 1024;     // bytes of the device DF-SANE state (V_DFS)

// surface buffers [N2][N1]
enum { S_P = 0, S_POLD, S_T, S_G, S_U, S_R, S_H, S_H0, S_DU, S_DUPREV, S_TPREV, S_DT, S_NSURF };
// volume buffers [Nz][6][N2][N1] and the scalar field [Nz][N2][N1]
enum { V_X = S_NSURF, V_F, V_XT, V_FT, V_B, V_DEP, V_TMP, V_DE, V_EP, V_PART, V_WZ, V_PKS, V_DFS, V_END };
static_assert(V_END <= FVIM_NSOLVER_BUFS, "workspace slots");

template <typename T> size_t esz() { return sizeof(T); }

template <typename T> int ensure_ws(fvim_ctx* c) {
  if (c->sv[V_PART]) return FVIM_OK;
  const size_t ns = (size_t)c->n1 * c->n2, nv = ns * c->nz;
  for (int i = 0; i < S_NSURF; ++i)
    if (FVIM_CU(cudaMalloc(&c->sv[i], ns * sizeof(T)))) return FVIM_ERR_OOM;
  for (int i = V_X; i <= V_DE; ++i)
    if (FVIM_CU(cudaMalloc(&c->sv[i], nv * 6 * sizeof(T)))) return FVIM_ERR_OOM;
  if (FVIM_CU(cudaMalloc(&c->sv[V_EP], nv * sizeof(T)))) return FVIM_ERR_OOM;
  if (FVIM_CU(cudaMalloc(&c->sv[V_PART], (size_t)RMAXB * NVMAX * sizeof(double)))) return FVIM_ERR_OOM;
  if (FVIM_CU(cudaMalloc(&c->sv[V_WZ], (size_t)c->nz * sizeof(double)))) return FVIM_ERR_OOM;
  if (FVIM_CU(cudaMalloc(&c->sv[V_PKS], kScalarBlock))) return FVIM_ERR_OOM;
  if (FVIM_CU(cudaMalloc(&c->sv[V_DFS], kDfsBytes))) return FVIM_ERR_OOM;
  if (FVIM_CU(cudaMallocHost(&c->h_part, (size_t)RMAXB * NVMAX * sizeof(double) + 256 + kDfsBytes))) {
    c->h_part = nullptr;
    return FVIM_ERR_OOM;
  }
  // trapezoid weights of the depth nodes times the cell area dA (discrete L2 product)
  std::vector<double> wz(c->nz, 0.0);
  const double dA = c->L1 * c->L2 / (double)ns;
  for (int i = 0; i + 1 < c->nz; ++i) {
    const double h = c->z_host[i + 1] - c->z_host[i];
    wz[i] += 0.5 * h * dA;
    wz[i + 1] += 0.5 * h * dA;
  }
  if (FVIM_CU(cudaMemcpy(c->sv[V_WZ], wz.data(), c->nz * sizeof(double), cudaMemcpyHostToDevice)))
    return FVIM_ERR_CUDA;
  for (int i = 0; i < V_PART; ++i)
    if (FVIM_CU(cudaMemset(c->sv[i], 0, (i < S_NSURF ? ns : (i == V_EP ? nv : nv * 6)) * sizeof(T))))
      return FVIM_ERR_CUDA;
  return FVIM_OK;
}

template <typename T> T* S(fvim_ctx* c, int i) { return (T*)c->sv[i]; }

// ---- solver runtime: an own non-blocking stream (so that the solver loops can be captured
// into CUDA graphs whatever stream the caller uses) and the captured graphs ---------------
struct GraphKey {
  const void* ptr[3];
  double d[2];
  int i;
  bool operator==(const GraphKey& o) const {
    return ptr[0] == o.ptr[0] && ptr[1] == o.ptr[1] && ptr[2] == o.ptr[2] && d[0] == o.d[0] && d[1] == o.d[1] &&
           i == o.i;
  }
};
struct SolverRT {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<std::pair<GraphKey, cudaGraphExec_t>> cg, df;  // CG batches, residual evaluations
  std::vector<std::pair<GraphKey, cudaGraphExec_t>> cgw;     // device CG loops (WHILE node)
  cudaGraphExec_t dfloop = nullptr;                          // device DF-SANE loop (WHILE node)
  bool dfloop_failed = false;                                // building it failed: host loop
  bool cgw_failed = false;                                   // building a CG loop failed: host loop
};
constexpr size_t kMaxGraphs = 8;

static void drop(std::vector<std::pair<GraphKey, cudaGraphExec_t>>& v) {
  for (auto& e : v) cudaGraphExecDestroy(e.second);
  v.clear();
}

static SolverRT* rt(fvim_ctx* c) {
  if (c->srt) return (SolverRT*)c->srt;
  SolverRT* r = new (std::nothrow) SolverRT();
  if (!r) return nullptr;
  if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (r->stream) cudaStreamDestroy(r->stream);
    if (r->ev_in) cudaEventDestroy(r->ev_in);
    delete r;
    return nullptr;
  }
  c->srt = r;
  return r;
}

// Runs body() (a fixed launch sequence on c->stream) through a CUDA graph captured on first
// use for this key; launches it directly while kernels are being timed one by one, when
// FVIM_SOLVER_GRAPHS=0, and whenever capture, instantiation or a graph launch fails.
static bool graphs_enabled() {
  static const bool on = [] {
    const char* e = getenv("FVIM_SOLVER_GRAPHS");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <class F>
static int graph_run(fvim_ctx* c, std::vector<std::pair<GraphKey, cudaGraphExec_t>>& cache, const GraphKey& key,
                     F&& body) {
  if (c->prof || !graphs_enabled()) return body();
  for (auto& e : cache)
    if (e.first == key) {
      if (!FVIM_CU(cudaGraphLaunch(e.second, c->stream))) return FVIM_OK;
      cudaGetLastError();
      return body();
    }
  if (FVIM_CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal))) {
    cudaGetLastError();
    return body();
  }
  const int rc = body();
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
  if (FVIM_CU(ce) || !g) {
    // the capture was invalidated (nothing ran): issue the sequence directly
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return body();
  }
  if (rc != FVIM_OK) {
    cudaGraphDestroy(g);
    return rc;
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (FVIM_CU(ie)) {
    cudaGetLastError();
    return body();
  }
  if (cache.size() >= kMaxGraphs) {
    cudaGraphExecDestroy(cache.front().second);
    cache.erase(cache.begin());
  }
  cache.emplace_back(key, ex);
  if (!FVIM_CU(cudaGraphLaunch(ex, c->stream))) return FVIM_OK;
  cudaGetLastError();
  return body();
}

// The solver entry points run on the runtime's stream, ordered after the caller's stream
// by an event on entry, and the caller's stream waits for them on exit.
struct OnSolverStream {
  fvim_ctx* c;
  cudaStream_t user;
  SolverRT* r;
  explicit OnSolverStream(fvim_ctx* ctx) : c(ctx), user(ctx->stream), r(rt(ctx)) {
    if (r && cudaEventRecord(r->ev_in, user) == cudaSuccess && cudaStreamWaitEvent(r->stream, r->ev_in, 0) == cudaSuccess)
      c->stream = r->stream;
    else
      r = nullptr;
  }
  ~OnSolverStream() {
    if (!r) return;
    cudaEventRecord(r->ev_out, r->stream);
    cudaStreamWaitEvent(user, r->ev_out, 0);
    c->stream = user;
  }
};


// Builds a graph of one WHILE conditional node whose body is what body(cond) launches on
// c->stream (captured); the body sets the loop condition through cond.  The condition starts
// at 1, so the body runs at least once.
template <class F> static int build_while_graph(fvim_ctx* c, F&& body, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  if (FVIM_CU(cudaGraphCreate(&g, 0))) return FVIM_ERR_CUDA;
  cudaGraphConditionalHandle cond;
  alignas(cudaGraphNodeParams) unsigned char cpbuf[sizeof(cudaGraphNodeParams)];
  memset(cpbuf, 0, sizeof(cpbuf));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cpbuf);
  cudaGraphNode_t node;
  if (FVIM_CU(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault))) {
    cudaGraphDestroy(g);
    return FVIM_ERR_CUDA;
  }
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (FVIM_CU(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp))) {
    cudaGraphDestroy(g);
    return FVIM_ERR_CUDA;
  }
  cudaGraph_t bg = cp.conditional.phGraph_out[0];
  if (FVIM_CU(cudaStreamBeginCaptureToGraph(c->stream, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal))) {
    cudaGraphDestroy(g);
    return FVIM_ERR_CUDA;
  }
  const int rc = body(cond);
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c->stream, &captured);
  if (rc != FVIM_OK || FVIM_CU(ce)) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return rc != FVIM_OK ? rc : FVIM_ERR_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (FVIM_CU(ie)) {
    cudaGetLastError();
    return FVIM_ERR_CUDA;
  }
  *out = ex;
  return FVIM_OK;
}

// ---- block reduction of NV doubles into partial[blockIdx.x][NV] -------------------
template <int NV> __device__ __forceinline__ void block_reduce(double (&v)[NV], double* partial) {
  __shared__ double sh[NV][RT / 32];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double x = v[j];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sh[j][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = 0;
      for (int w = 0; w < RT / 32; ++w) s += sh[j][w];
      partial[blockIdx.x * NV + j] = s;
    }
  }
}

inline int rgrid(size_t n) {
  size_t b = (n + RT - 1) / RT;
  return (int)std::min<size_t>(std::max<size_t>(b, 1), RMAXB);
}

// copy the partials of a reduction grid and add them in block order
template <int NV> int finish(fvim_ctx* c, int nblk, double* out) {
  if (FVIM_CU(cudaMemcpyAsync(c->h_part, c->sv[V_PART], (size_t)nblk * NV * sizeof(double), cudaMemcpyDeviceToHost,
                      c->stream)))
    return FVIM_ERR_CUDA;
  if (FVIM_CU(cudaStreamSynchronize(c->stream))) return FVIM_ERR_CUDA;
  for (int j = 0; j < NV; ++j) out[j] = 0;
  for (int b = 0; b < nblk; ++b)
    for (int j = 0; j < NV; ++j) out[j] += c->h_part[b * NV + j];
  return FVIM_OK;
}

// ---- Polonsky-Keer kernels (surface, n = N1 N2) ------------------------------------
// sum over the contact set of u - h, and its size
template <typename T>
__global__ void k_pk_stats(const T* __restrict__ u, const T* __restrict__ h, const T* __restrict__ p, size_t n,
                           double* part) {
  double v[2] = {0, 0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
    if (p[i] > 0) { v[0] += (double)u[i] - (double)h[i]; v[1] += 1; }
  block_reduce<2>(v, part);
}
// g = u - h - gbar; sum over the contact set of g^2
template <typename T>
__global__ void k_pk_g(const T* __restrict__ u, const T* __restrict__ h, const T* __restrict__ p, T* __restrict__ g,
                       double gbar, size_t n, double* part) {
  double v[1] = {0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    const T gi = (T)((double)u[i] - (double)h[i] - gbar);
    g[i] = gi;
    if (p[i] > 0) v[0] += (double)gi * (double)gi;
  }
  block_reduce<1>(v, part);
}
// conjugate direction t = g + beta t on the contact set, 0 elsewhere
template <typename T>
__global__ void k_pk_dir(const T* __restrict__ g, const T* __restrict__ p, T* __restrict__ t, double beta, size_t n) {
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
    t[i] = p[i] > 0 ? (T)((double)g[i] + beta * (double)t[i]) : (T)0;
}
// sum over the contact set of r
template <typename T>
__global__ void k_pk_rsum(const T* __restrict__ r, const T* __restrict__ p, size_t n, double* part) {
  double v[1] = {0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
    if (p[i] > 0) v[0] += (double)r[i];
  block_reduce<1>(v, part);
}
// <g, t> and <r - rbar, t> over the contact set
template <typename T>
__global__ void k_pk_dots(const T* __restrict__ g, const T* __restrict__ t, const T* __restrict__ r,
                          const T* __restrict__ p, double rbar, size_t n, double* part) {
  double v[2] = {0, 0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
    if (p[i] > 0) {
      v[0] += (double)g[i] * (double)t[i];
      v[1] += ((double)r[i] - rbar) * (double)t[i];
    }
  block_reduce<2>(v, part);
}
// p <- max(p - tau t, 0); penetrating points with zero pressure get -tau g
template <typename T>
__global__ void k_pk_update(T* __restrict__ p, T* __restrict__ pold, const T* __restrict__ t,
                            const T* __restrict__ g, double tau, size_t n, double* part) {
  double v[2] = {0, 0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    const T po = p[i];
    T pn = (T)fmax((double)po - tau * (double)t[i], 0.0);
    const bool ol = (pn == (T)0) && (g[i] < (T)0);
    if (ol) pn = (T)(-tau * (double)g[i]);
    pold[i] = po;
    p[i] = pn;
    v[0] += (double)pn;
    v[1] += ol ? 1.0 : 0.0;
  }
  block_reduce<2>(v, part);
}
// p <- s p; sum |p - p_old| and the size of the contact set
template <typename T>
__global__ void k_pk_scale(T* __restrict__ p, const T* __restrict__ pold, double s, size_t n, double* part) {
  double v[2] = {0, 0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    const T pn = (T)(s * (double)p[i]);
    p[i] = pn;
    v[0] += fabs((double)pn - (double)pold[i]);
    v[1] += pn > (T)0 ? 1.0 : 0.0;
  }
  block_reduce<2>(v, part);
}
template <typename T> __global__ void k_fill(T* __restrict__ a, T v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) a[i] = v;
}
// sum of a and of a^2
template <typename T> __global__ void k_sum2(const T* __restrict__ a, size_t n, double* part) {
  double v[2] = {0, 0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    v[0] += (double)a[i];
    v[1] += (double)a[i] * (double)a[i];
  }
  block_reduce<2>(v, part);
}
// c = a + s b (elementwise)
template <typename T>
__global__ void k_axpby(T* __restrict__ cc, const T* __restrict__ a, double s, const T* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
    cc[i] = (T)((double)a[i] + s * (double)b[i]);
}
// ||a - b||^2
template <typename T>
__global__ void k_diff2(const T* __restrict__ a, const T* __restrict__ b, size_t n, double* part) {
  double v[1] = {0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    const double d = (double)a[i] - (double)b[i];
    v[0] += d * d;
  }
  block_reduce<1>(v, part);
}

// Algorithm 1: relaxed = dU_prev + lambda (dU - dU_prev); H = H0 - relaxed; then dU_prev = dU
// (the listing's order, carry = 0) or dU_prev = relaxed (under-relaxation that carries the
// relaxed value, carry = 1)
template <typename T>
__global__ void k_relax(T* __restrict__ H, const T* __restrict__ H0, T* __restrict__ dUp, const T* __restrict__ dU,
                        double lam, int carry, size_t n) {
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    const double relaxed = (double)dUp[i] + lam * ((double)dU[i] - (double)dUp[i]);
    H[i] = (T)((double)H0[i] - relaxed);
    dUp[i] = carry ? (T)relaxed : dU[i];
  }
}
// number of positive entries
template <typename T> __global__ void k_count_pos(const T* __restrict__ a, size_t n, double* part) {
  double v[1] = {0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
    v[0] += a[i] > (T)0 ? 1.0 : 0.0;
  block_reduce<1>(v, part);
}

// ---- DF-SANE kernels (volume [Nz][6][N2][N1], weighted L2 product) ------------------
// Plane zc = (z, c) of the volume has the trapezoid weight dA w_z, doubled for the three
// shear components.  N1 N2 is a power of two, so the plane of an index is a shift.  FP32
// vectors are processed four values at a time: the four products are summed in FP32 and
// the partial is accumulated in FP64 (one FP64 multiply-add per four values); FP64
// vectors keep every operation in FP64.
__device__ __forceinline__ double plane_weight(const double* wz, unsigned zc) {
  return wz[zc / 6] * ((zc % 6) < 3 ? 1.0 : 2.0);
}

// F = x - b - tmp ; <F, F>
template <typename T>
__global__ void k_df_res(const T* __restrict__ x, const T* __restrict__ b, const T* __restrict__ tmp,
                         T* __restrict__ F, const double* __restrict__ wz, int lgxy, size_t n, double* part) {
  double v[1] = {0};
  if constexpr (sizeof(T) == 4) {
    const size_t n4 = n >> 2;
    const int lg4 = lgxy - 2;
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n4; i += (size_t)gridDim.x * RT) {
      const float4 a = reinterpret_cast<const float4*>(x)[i];
      const float4 c = reinterpret_cast<const float4*>(b)[i];
      const float4 d = reinterpret_cast<const float4*>(tmp)[i];
      const float4 f = make_float4(a.x - c.x - d.x, a.y - c.y - d.y, a.z - c.z - d.z, a.w - c.w - d.w);
      reinterpret_cast<float4*>(F)[i] = f;
      const float q = f.x * f.x + f.y * f.y + f.z * f.z + f.w * f.w;
      v[0] += plane_weight(wz, (unsigned)(i >> lg4)) * (double)q;
    }
  } else {
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
      const T f = x[i] - b[i] - tmp[i];
      F[i] = f;
      v[0] += plane_weight(wz, (unsigned)(i >> lgxy)) * (double)f * (double)f;
    }
  }
  block_reduce<1>(v, part);
}
// <s, s> and <s, y> with s = xn - x, y = Fn - F
template <typename T>
__global__ void k_df_sy(const T* __restrict__ x, const T* __restrict__ xn, const T* __restrict__ F,
                        const T* __restrict__ Fn, const double* __restrict__ wz, int lgxy, size_t n, double* part) {
  double v[2] = {0, 0};
  if constexpr (sizeof(T) == 4) {
    const size_t n4 = n >> 2;
    const int lg4 = lgxy - 2;
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n4; i += (size_t)gridDim.x * RT) {
      const float4 a = reinterpret_cast<const float4*>(x)[i];
      const float4 an = reinterpret_cast<const float4*>(xn)[i];
      const float4 f = reinterpret_cast<const float4*>(F)[i];
      const float4 fn = reinterpret_cast<const float4*>(Fn)[i];
      const float s0 = an.x - a.x, s1 = an.y - a.y, s2 = an.z - a.z, s3 = an.w - a.w;
      const float y0 = fn.x - f.x, y1 = fn.y - f.y, y2 = fn.z - f.z, y3 = fn.w - f.w;
      const double w = plane_weight(wz, (unsigned)(i >> lg4));
      v[0] += w * (double)(s0 * s0 + s1 * s1 + s2 * s2 + s3 * s3);
      v[1] += w * (double)(s0 * y0 + s1 * y1 + s2 * y2 + s3 * y3);
    }
  } else {
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
      const double w = plane_weight(wz, (unsigned)(i >> lgxy));
      const double s = (double)xn[i] - (double)x[i];
      const double y = (double)Fn[i] - (double)F[i];
      v[0] += w * s * s;
      v[1] += w * s * y;
    }
  }
  block_reduce<2>(v, part);
}
// dst = a + s b over a volume vector (FP32: four values at a time, FP32 arithmetic)
template <typename T>
__global__ void k_axpby_vol(T* __restrict__ dst, const T* __restrict__ a, double s, const double* __restrict__ sdev,
                            const T* __restrict__ b, size_t n) {
  if (sdev) s *= *sdev;
  if constexpr (sizeof(T) == 4) {
    const float sf = (float)s;
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < (n >> 2); i += (size_t)gridDim.x * RT) {
      const float4 x = reinterpret_cast<const float4*>(a)[i];
      const float4 y = reinterpret_cast<const float4*>(b)[i];
      reinterpret_cast<float4*>(dst)[i] =
          make_float4(fmaf(sf, y.x, x.x), fmaf(sf, y.y, x.y), fmaf(sf, y.z, x.z), fmaf(sf, y.w, x.w));
    }
  } else {
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) dst[i] = a[i] + s * b[i];
  }
}

template <typename T> int sum2(fvim_ctx* c, const T* a, size_t n, double* out) {
  const int g = rgrid(n);
  k_sum2<T><<<g, RT, 0, c->stream>>>(a, n, (double*)c->sv[V_PART]);
  FVIM_CUDA_CHECK_LAUNCH();
  return finish<2>(c, g, out);
}

template <typename T> int axpby(fvim_ctx* c, T* dst, const T* a, double s, const T* b, size_t n) {
  k_axpby<T><<<rgrid(n), RT, 0, c->stream>>>(dst, a, s, b, n);
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}
// dst = a + s (*sdev) b (sdev: a device scalar, or NULL for 1)
template <typename T>
int axpby_vol(fvim_ctx* c, T* dst, const T* a, double s, const double* sdev, const T* b, size_t n) {
  k_axpby_vol<T><<<rgrid(sizeof(T) == 4 ? n / 4 : n), RT, 0, c->stream>>>(dst, a, s, sdev, b, n);
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

// surface displacement u = K*p of the Boussinesq operator (u3_hat = 2 p_hat / (E* q))
template <typename T> int conv(fvim_ctx* c, const T* p, T* u) { return apply_boussinesq_t<T>(c, p, u, nullptr, FVIM_STRAIN); }

// ---- Polonsky-Keer constrained conjugate gradient ----------------------------------
// The scalars of an iteration live on the device (PKS); every reduction is finished by a
// one-block kernel that also applies the scalar logic, so an iteration is a fixed launch
// sequence without host round trips.  Once the stop test has fired (or a non-finite value
// appeared) the update kernels return at entry, so iterations issued after convergence
// leave the pressure untouched: the host only reads the flag every few iterations.
struct PKS {
  double nIc, gbar, G_old, beta, delta, rbar, tau, s, err;
  int done, it, bad, passes;  // passes: WHILE-loop passes of the device CG loop
};
static_assert(sizeof(PKS) <= 128, "the DF-SANE step is kept at byte 128 of the scalar block");

// layer range [zr[0], zr[1]) of the voxels that flow in the last return map (byte 200 of the
// scalar block), reset before each return map; the Mindlin apply of the plastic strain
// increment skips the forward transforms of the other layers, where the increment is zero
// (the layer-level form of the sparse plastic support noted in Sec. 3.2)
static_assert(200 + 2 * sizeof(int) <= kScalarBlock, "flow range inside the scalar block");
inline int* flow_range(fvim_ctx* c) { return reinterpret_cast<int*>(static_cast<char*>(c->sv[V_PKS]) + 200); }
inline int reset_flow_range(fvim_ctx* c) {
  int* zr = flow_range(c);
  if (FVIM_CU(cudaMemsetAsync(zr, 0x7f, sizeof(int), c->stream)) ||
      FVIM_CU(cudaMemsetAsync(zr + 1, 0, sizeof(int), c->stream)))
    return FVIM_ERR_CUDA;
  return FVIM_OK;
}

// sum the partials [nblk][NV] of a reduction grid in a fixed order (one block)
template <int NV> __device__ __forceinline__ void fin_sum(const double* part, int nblk, double (&out)[NV]) {
  __shared__ double sh[NV][RT];
  double v[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = 0;
  for (int b = threadIdx.x; b < nblk; b += RT)
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] += __ldcg(part + b * NV + j);
#pragma unroll
  for (int j = 0; j < NV; ++j) sh[j][threadIdx.x] = v[j];
  __syncthreads();
  for (int w = RT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int j = 0; j < NV; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = sh[j][0];
}

__device__ __forceinline__ void fin_stats(const double* part, int nblk, PKS* S) {
  if (S->done) return;
  double v[2];
  fin_sum<2>(part, nblk, v);
  if (threadIdx.x == 0) {
    S->nIc = v[1];
    if (!(v[1] > 0) || !isfinite(v[0])) { S->bad = 1; S->done = 1; }
    else S->gbar = v[0] / v[1];
  }
}
__device__ __forceinline__ void fin_G(const double* part, int nblk, PKS* S) {
  if (S->done) return;
  double v[1];
  fin_sum<1>(part, nblk, v);
  if (threadIdx.x == 0) {
    S->beta = S->delta * (v[0] / S->G_old);
    S->G_old = v[0];
  }
}
__device__ __forceinline__ void fin_rbar(const double* part, int nblk, PKS* S) {
  if (S->done) return;
  double v[1];
  fin_sum<1>(part, nblk, v);
  if (threadIdx.x == 0) S->rbar = v[0] / S->nIc;
}
__device__ __forceinline__ void fin_tau(const double* part, int nblk, PKS* S) {
  if (S->done) return;
  double v[2];
  fin_sum<2>(part, nblk, v);
  if (threadIdx.x == 0) S->tau = v[1] != 0 ? v[0] / v[1] : 0.0;
}
__device__ __forceinline__ void fin_scale(const double* part, int nblk, PKS* S, double W, double dA) {
  if (S->done) return;
  double v[2];
  fin_sum<2>(part, nblk, v);
  if (threadIdx.x == 0) {
    S->delta = v[1] > 0 ? 0.0 : 1.0;
    if (!(v[0] > 0) || !isfinite(v[0])) { S->bad = 1; S->done = 1; }
    else S->s = W / (dA * v[0]);
  }
}
__device__ __forceinline__ void fin_err(const double* part, int nblk, PKS* S, double W, double dA, double tol, int max_it) {
  if (S->done) return;
  double v[2];
  fin_sum<2>(part, nblk, v);
  if (threadIdx.x == 0) {
    S->err = dA * v[0] / W;
    S->it += 1;
    if (S->err < tol || S->it >= max_it) S->done = 1;
    if (!isfinite(S->err)) { S->bad = 1; S->done = 1; }
  }
}

// The reduction kernels below finish their own sums: the last block to arrive (counted
// with an atomic, after a fence) adds the partials in block order and applies the scalar
// logic, then re-arms the counter for the next kernel.
__device__ __forceinline__ bool last_block(unsigned* cnt) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}
__device__ __forceinline__ void rearm(unsigned* cnt) {
  if (threadIdx.x == 0) *cnt = 0u;
}

template <typename T>
__global__ void k_pkd_stats(const T* __restrict__ u, const T* __restrict__ h, const T* __restrict__ p, size_t n,
                            double* part, PKS* S, unsigned* cnt) {
  if (S->done) return;
  double v[2] = {0, 0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
    if (p[i] > 0) { v[0] += (double)u[i] - (double)h[i]; v[1] += 1; }
  block_reduce<2>(v, part);
  if (last_block(cnt)) {
    fin_stats(part, gridDim.x, S);
    rearm(cnt);
  }
}
template <typename T>
__global__ void k_pkd_g(const T* __restrict__ u, const T* __restrict__ h, const T* __restrict__ p, T* __restrict__ g,
                        size_t n, double* part, PKS* S, unsigned* cnt) {
  if (S->done) return;
  const double gbar = S->gbar;
  double v[1] = {0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    const T gi = (T)((double)u[i] - (double)h[i] - gbar);
    g[i] = gi;
    if (p[i] > 0) v[0] += (double)gi * (double)gi;
  }
  block_reduce<1>(v, part);
  if (last_block(cnt)) {
    fin_G(part, gridDim.x, S);
    rearm(cnt);
  }
}
template <typename T>
__global__ void k_pkd_dir(const T* __restrict__ g, const T* __restrict__ p, T* __restrict__ t, size_t n,
                          const PKS* S) {
  if (S->done) return;
  const double beta = S->beta;
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
    t[i] = p[i] > 0 ? (T)((double)g[i] + beta * (double)t[i]) : (T)0;
}
template <typename T>
__global__ void k_pkd_rsum(const T* __restrict__ r, const T* __restrict__ p, size_t n, double* part, PKS* S,
                           unsigned* cnt) {
  if (S->done) return;
  double v[1] = {0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
    if (p[i] > 0) v[0] += (double)r[i];
  block_reduce<1>(v, part);
  if (last_block(cnt)) {
    fin_rbar(part, gridDim.x, S);
    rearm(cnt);
  }
}
template <typename T>
__global__ void k_pkd_dots(const T* __restrict__ g, const T* __restrict__ t, const T* __restrict__ r,
                           const T* __restrict__ p, size_t n, double* part, PKS* S, unsigned* cnt) {
  if (S->done) return;
  const double rbar = S->rbar;
  double v[2] = {0, 0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
    if (p[i] > 0) {
      v[0] += (double)g[i] * (double)t[i];
      v[1] += ((double)r[i] - rbar) * (double)t[i];
    }
  block_reduce<2>(v, part);
  if (last_block(cnt)) {
    fin_tau(part, gridDim.x, S);
    rearm(cnt);
  }
}
template <typename T>
__global__ void k_pkd_update(T* __restrict__ p, T* __restrict__ pold, const T* __restrict__ t,
                             const T* __restrict__ g, size_t n, double* part, PKS* S, unsigned* cnt, double W,
                             double dA) {
  if (S->done) return;
  const double tau = S->tau;
  double v[2] = {0, 0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    const T po = p[i];
    T pn = (T)fmax((double)po - tau * (double)t[i], 0.0);
    const bool ol = (pn == (T)0) && (g[i] < (T)0);
    if (ol) pn = (T)(-tau * (double)g[i]);
    pold[i] = po;
    p[i] = pn;
    v[0] += (double)pn;
    v[1] += ol ? 1.0 : 0.0;
  }
  block_reduce<2>(v, part);
  if (last_block(cnt)) {
    fin_scale(part, gridDim.x, S, W, dA);
    rearm(cnt);
  }
}
template <typename T>
__global__ void k_pkd_scale(T* __restrict__ p, const T* __restrict__ pold, size_t n, double* part, PKS* S,
                            unsigned* cnt, double W, double dA, double tol, int max_it) {
  if (S->done) return;
  const double s = S->s;
  double v[2] = {0, 0};
  for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
    const T pn = (T)(s * (double)p[i]);
    p[i] = pn;
    v[0] += fabs((double)pn - (double)pold[i]);
    v[1] += pn > (T)0 ? 1.0 : 0.0;
  }
  block_reduce<2>(v, part);
  if (last_block(cnt)) {
    fin_err(part, gridDim.x, S, W, dA, tol, max_it);
    rearm(cnt);
  }
}

// loop condition of the device CG loop (one thread): stop when the iteration logic has set
// the stop flag, and after max_it passes in any case, so that the loop always ends
__global__ void k_pkd_cond(PKS* S, int max_it, cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  S->passes += 1;
  cudaGraphSetConditional(cond, (S->done || S->passes >= max_it) ? 0u : 1u);
}

// the CG iterations run as one WHILE graph unless FVIM_DEVICE_CG=0 (read on every solve)
static bool device_cg_enabled() {
  const char* e = getenv("FVIM_DEVICE_CG");
  return !(e && e[0] == '0');
}

template <typename T>
int elastic_contact_t(fvim_ctx* c, const T* h, double W, T* p, const fvim_opts* o, int* iters, double* err_out) {
  const size_t n = (size_t)c->n1 * c->n2;
  const double dA = c->L1 * c->L2 / (double)n;
  double* part = (double*)c->sv[V_PART];
  PKS* st = (PKS*)c->sv[V_PKS];
  T *pold = S<T>(c, S_POLD), *t = S<T>(c, S_T), *g = S<T>(c, S_G), *u = S<T>(c, S_U), *r_ = S<T>(c, S_R);
  const int grd = rgrid(n);
  double v[2];
  int rc;
  // initial pressure: the given guess scaled to the load, or uniform
  if ((rc = sum2<T>(c, p, n, v))) return rc;
  if (v[0] > 0) {
    k_axpby<T><<<grd, RT, 0, c->stream>>>(p, p, W / (dA * v[0]) - 1.0, p, n);
  } else {
    k_fill<T><<<grd, RT, 0, c->stream>>>(p, (T)(W / (c->L1 * c->L2)), n);
  }
  k_fill<T><<<grd, RT, 0, c->stream>>>(t, (T)0, n);
  FVIM_CUDA_CHECK_LAUNCH();
  PKS s0;
  memset(&s0, 0, sizeof(s0));
  s0.G_old = 1.0;
  s0.err = INFINITY;
  if (FVIM_CU(cudaMemcpyAsync(st, &s0, sizeof(PKS), cudaMemcpyHostToDevice, c->stream))) return FVIM_ERR_CUDA;
  // arrival counter of the self-finishing reductions (byte 192 of the scalar block)
  unsigned* cnt = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(st) + 192);
  if (FVIM_CU(cudaMemsetAsync(cnt, 0, sizeof(unsigned), c->stream))) return FVIM_ERR_CUDA;
  PKS* sh = reinterpret_cast<PKS*>(c->h_part + (size_t)RMAXB * NVMAX);  // pinned
  *sh = s0;
  SolverRT* srt = rt(c);
  const GraphKey key{{h, p, nullptr}, {W, o->cg_tol}, o->cg_max_iter};
  auto one_iteration = [&]() -> int {
    int r;
    if ((r = conv<T>(c, p, u))) return r;
    k_pkd_stats<T><<<grd, RT, 0, c->stream>>>(u, h, p, n, part, st, cnt);
    k_pkd_g<T><<<grd, RT, 0, c->stream>>>(u, h, p, g, n, part, st, cnt);
    k_pkd_dir<T><<<grd, RT, 0, c->stream>>>(g, p, t, n, st);
    if ((r = conv<T>(c, t, r_))) return r;
    k_pkd_rsum<T><<<grd, RT, 0, c->stream>>>(r_, p, n, part, st, cnt);
    k_pkd_dots<T><<<grd, RT, 0, c->stream>>>(g, t, r_, p, n, part, st, cnt);
    k_pkd_update<T><<<grd, RT, 0, c->stream>>>(p, pold, t, g, n, part, st, cnt, W, dA);
    k_pkd_scale<T><<<grd, RT, 0, c->stream>>>(p, pold, n, part, st, cnt, W, dA, o->cg_tol, o->cg_max_iter);
    FVIM_CUDA_CHECK_LAUNCH();
    return FVIM_OK;
  };
  // the iterations as one WHILE graph per (surface, pressure, load, tolerance, cap): one
  // iteration and the loop condition per pass, one read of the state at the end
  bool ran_device = false;
  if (srt && !c->prof && graphs_enabled() && device_cg_enabled() && o->cg_max_iter > 0) {
    cudaGraphExec_t ex = nullptr;
    for (auto& e : srt->cgw)
      if (e.first == key) ex = e.second;
    if (!ex && !srt->cgw_failed) {
      const int max_it = o->cg_max_iter;
      const int b = build_while_graph(
          c,
          [&](cudaGraphConditionalHandle cond) -> int {
            int r;
            if ((r = one_iteration())) return r;
            k_pkd_cond<<<1, 32, 0, c->stream>>>(st, max_it, cond);
            FVIM_CUDA_CHECK_LAUNCH();
            return FVIM_OK;
          },
          &ex);
      if (b == FVIM_OK) {
        if (srt->cgw.size() >= kMaxGraphs) {
          cudaGraphExecDestroy(srt->cgw.front().second);
          srt->cgw.erase(srt->cgw.begin());
        }
        srt->cgw.emplace_back(key, ex);
      } else {
        srt->cgw_failed = true;  // the host loop below takes over
        ex = nullptr;
        cudaGetLastError();
      }
    }
    if (ex) {
      if (FVIM_CU(cudaGraphLaunch(ex, c->stream)) ||
          FVIM_CU(cudaMemcpyAsync(sh, st, sizeof(PKS), cudaMemcpyDeviceToHost, c->stream)) ||
          FVIM_CU(cudaStreamSynchronize(c->stream)))
        return FVIM_ERR_CUDA;
      ran_device = true;
    }
  }
  const int batch = 4;  // iterations issued between two reads of the stop flag
  for (int issued = 0; !ran_device && issued < o->cg_max_iter;) {
    const int nb = std::min(batch, o->cg_max_iter - issued);
    auto iterations = [&]() -> int {
      int r;
      for (int b = 0; b < nb; ++b)
        if ((r = one_iteration())) return r;
      return FVIM_OK;
    };
    // a full batch is one captured graph per (surface, pressure, load, tolerance)
    if ((rc = (nb == batch && srt) ? graph_run(c, srt->cg, key, iterations) : iterations())) return rc;
    issued += nb;
    if (FVIM_CU(cudaMemcpyAsync(sh, st, sizeof(PKS), cudaMemcpyDeviceToHost, c->stream))) return FVIM_ERR_CUDA;
    if (FVIM_CU(cudaStreamSynchronize(c->stream))) return FVIM_ERR_CUDA;
    if (sh->done) break;
  }
  if (sh->bad) return FVIM_ERR_NONFINITE;
  if (iters) *iters = sh->it;
  if (err_out) *err_out = sh->err;
  return sh->err < o->cg_tol ? FVIM_OK : FVIM_ERR_NOT_CONVERGED;
}

// ---- DF-SANE on R[x] = x - b - grad^sym N[C:deps_p(x; S)] --------------------------
// spectral step sigma = <s, s> / <s, y> with its safeguard, finished on the device so the
// next trial point needs no host round trip
__global__ void k_df_sigma(const double* part, int nblk, double fn, double smin, double smax, double* sig) {
  double v[2];
  fin_sum<2>(part, nblk, v);
  if (threadIdx.x == 0) {
    double sigma = v[1] != 0 ? v[0] / v[1] : INFINITY;
    if (!(fabs(sigma) >= smin && fabs(sigma) <= smax)) {
      const double nf = sqrt(fn);
      sigma = nf > 1 ? 1.0 : (nf >= 1e-5 ? 1.0 / nf : 1e5);
    }
    *sig = sigma;
  }
}
__global__ void k_set_double(double* d, double v) { *d = v; }

template <typename T> struct DF {
  fvim_ctx* c;
  size_t n, nxy;
  int grd;
  int lgxy;  // log2(N1 N2)
  // F(x) into Fx; returns ||F||^2 (weighted).  The launch sequence is one captured graph
  // per (x, Fx) pair.
  int eval(const T* x, T* Fx, double* f) {
    auto seq = [&]() -> int {
      int r;
      if ((r = reset_flow_range(c))) return r;
      if ((r = return_map_t<T>(c, x, S<T>(c, V_DEP), S<T>(c, V_EP), flow_range(c)))) return r;
      if ((r = apply_mindlin_t<T>(c, S<T>(c, V_DEP), S<T>(c, V_TMP), FVIM_STRAIN, nullptr, flow_range(c)))) return r;
      k_df_res<T><<<grd, RT, 0, c->stream>>>(x, S<T>(c, V_B), S<T>(c, V_TMP), Fx, (const double*)c->sv[V_WZ], lgxy,
                                            n, (double*)c->sv[V_PART]);
      FVIM_CUDA_CHECK_LAUNCH();
      return FVIM_OK;
    };
    SolverRT* srt = rt(c);
    const GraphKey key{{x, Fx, nullptr}, {0.0, 0.0}, 0};
    int rc = srt ? graph_run(c, srt->df, key, seq) : seq();
    if (rc) return rc;
    c->n_applies++;
    return finish<1>(c, grd, f);
  }
};

// ---- DF-SANE iterations on the device ---------------------------------------------------
// The loop below the initial evaluations runs as one CUDA graph: a WHILE node whose body is
// one trial evaluation (trial point, return map, Mindlin apply, residual norm, <s,s> and
// <s,y>) followed by a one-thread kernel that takes the host loop's decisions (accept the
// trial, try the opposite direction, shrink both steps, update sigma and the history, test
// convergence, stagnation and the caps) and sets the loop condition.  The current point and
// the trial point swap roles through pointers held in device memory.  Every decision uses the
// same formulas and FP64 values as the host loop; the trial count is capped, so the loop ends.
struct DFS {
  const void* px[2];  // the two point buffers: x = px[cur], trial = px[1 - cur]
  void* pF[2];        // their residuals
  double f, nF0, fmax, eta, ap, am, fp, fm, ftrial, best_old, tol_abs, tol_rel, gamma, smin, smax, tmin, tmax;
  double sy[2];
  double hist[32];    // ring of the accepted residuals, hist[i & 31] for i < len
  int len, k, bt, phase, done, conv, bad, cur, trials, max_iter, max_trials, evals;
};
static_assert(sizeof(DFS) <= kDfsBytes, "device DF-SANE state");
constexpr int kDfsM = 10, kDfsStag = 30;

// trial = x + coef F (coef = -ap sigma in phase 0, +am sigma in phase 1) fused with the return
// map at the trial point (Sec. 4.1, Sec. 4.3): one
// thread per voxel writes the trial point, the plastic strain increment and (d_ep not NULL)
// the increment of cumulated plastic strain, and notes the layer range of the flowing voxels.
// The loop leaves d_ep out: the solve recomputes the return map of its final point.
template <typename T>
__global__ void k_dfd_trial_rmap(const DFS* __restrict__ s, const double* __restrict__ dsig,
                                 const T* __restrict__ sig_n, const T* __restrict__ ep, T* __restrict__ d_eps_p,
                                 T* __restrict__ d_ep, size_t nxy, size_t nvox, T lam, T mu, T sy, T Eh,
                                 int* __restrict__ zr) {
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  const int cur = s->cur;
  const T* a = static_cast<const T*>(s->px[cur]);
  const T* b = static_cast<const T*>(s->pF[cur]);
  T* dst = const_cast<T*>(static_cast<const T*>(s->px[1 - cur]));
  const double coef = (s->phase == 0 ? -s->ap : s->am) * *dsig;
  const T cf = (T)coef;
  const size_t z = v / nxy, xy = v - z * nxy;
  const size_t base = z * 6 * nxy + xy;
  T de[6], sg[6], dp[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const size_t i = base + c * nxy;
    if constexpr (sizeof(T) == 4) de[c] = fmaf(cf, b[i], a[i]);
    else de[c] = fma(coef, (double)b[i], (double)a[i]);
    dst[i] = de[c];
    sg[c] = sig_n[i];
  }
  const T dEp = rmap_voxel(de, sg, ep[v], lam, mu, sy, Eh, dp);
#pragma unroll
  for (int c = 0; c < 6; ++c) d_eps_p[base + c * nxy] = dp[c];
  if (d_ep) d_ep[v] = dEp;
  if (dEp > 0) flow_range_note(zr, (int)z);
}

// residual of the trial point into its residual buffer, with ||F||^2 into s->ftrial and <s, s>,
// <s, y> (s = trial - x, y = F(trial) - F(x)) into s->sy (last block).  The trial point is
// recomputed from x and F with the expression the trial kernel wrote it with (the same
// values), so it is not read back.
template <typename T>
__global__ void k_dfd_res_sy(DFS* s, const double* __restrict__ dsig, const T* __restrict__ b,
                             const T* __restrict__ tmp, const double* __restrict__ wz, int lgxy, size_t n,
                             double* part, unsigned* cnt) {
  const int cur = s->cur;
  const T* x = static_cast<const T*>(s->px[cur]);
  const T* F = static_cast<const T*>(s->pF[cur]);
  T* Fn = static_cast<T*>(s->pF[1 - cur]);
  const double coef = (s->phase == 0 ? -s->ap : s->am) * *dsig;
  double v[3] = {0, 0, 0};
  if constexpr (sizeof(T) == 4) {
    const float cf = (float)coef;
    const size_t n4 = n >> 2;
    const int lg4 = lgxy - 2;
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n4; i += (size_t)gridDim.x * RT) {
      const float4 a = reinterpret_cast<const float4*>(x)[i];
      const float4 g = reinterpret_cast<const float4*>(F)[i];
      const float4 c = reinterpret_cast<const float4*>(b)[i];
      const float4 d = reinterpret_cast<const float4*>(tmp)[i];
      const float4 t = make_float4(fmaf(cf, g.x, a.x), fmaf(cf, g.y, a.y), fmaf(cf, g.z, a.z), fmaf(cf, g.w, a.w));
      const float4 f = make_float4(t.x - c.x - d.x, t.y - c.y - d.y, t.z - c.z - d.z, t.w - c.w - d.w);
      reinterpret_cast<float4*>(Fn)[i] = f;
      const double w = plane_weight(wz, (unsigned)(i >> lg4));
      const float q = f.x * f.x + f.y * f.y + f.z * f.z + f.w * f.w;
      v[0] += w * (double)q;
      const float s0 = t.x - a.x, s1 = t.y - a.y, s2 = t.z - a.z, s3 = t.w - a.w;
      const float y0 = f.x - g.x, y1 = f.y - g.y, y2 = f.z - g.z, y3 = f.w - g.w;
      v[1] += w * (double)(s0 * s0 + s1 * s1 + s2 * s2 + s3 * s3);
      v[2] += w * (double)(s0 * y0 + s1 * y1 + s2 * y2 + s3 * y3);
    }
  } else {
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
      const double w = plane_weight(wz, (unsigned)(i >> lgxy));
      const double xi = (double)x[i], gi = (double)F[i];
      const double t = fma(coef, gi, xi);
      const T f = (T)(t - (double)b[i] - (double)tmp[i]);
      Fn[i] = f;
      v[0] += w * (double)f * (double)f;
      const double a = t - xi;
      const double y = (double)f - gi;
      v[1] += w * a * a;
      v[2] += w * a * y;
    }
  }
  block_reduce<3>(v, part);
  if (last_block(cnt)) {
    double r[3];
    fin_sum<3>(part, gridDim.x, r);
    if (threadIdx.x == 0) {
      s->ftrial = r[0];
      s->sy[0] = r[1];
      s->sy[1] = r[2];
    }
    rearm(cnt);
  }
}

// the host loop's decisions after one trial evaluation (one thread)
__global__ void k_dfd_decide(DFS* s, double* dsig, cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  s->trials += 1;
  s->evals += 1;
  const double ft = s->ftrial;
  bool acc = false;
  if (s->phase == 0) {
    s->fp = ft;
    if (ft <= s->fmax + s->eta - s->gamma * s->ap * s->ap * s->f) acc = true;
    else s->phase = 1;
  } else {
    s->fm = ft;
    if (ft <= s->fmax + s->eta - s->gamma * s->am * s->am * s->f) {
      acc = true;
    } else {
      const double f = s->f, ap = s->ap, am = s->am;
      s->ap = fmin(fmax(ap * ap * f / (s->fp + (2 * ap - 1) * f), s->tmin * ap), s->tmax * ap);
      s->am = fmin(fmax(am * am * f / (s->fm + (2 * am - 1) * f), s->tmin * am), s->tmax * am);
      s->phase = 0;
      s->bt += 1;
      if (s->bt >= 60) s->done = 1;  // line search failed: stop, not converged
    }
  }
  if (acc) {
    double sigma = s->sy[1] != 0 ? s->sy[0] / s->sy[1] : INFINITY;
    if (!(fabs(sigma) >= s->smin && fabs(sigma) <= s->smax)) {
      const double nf = sqrt(ft);
      sigma = nf > 1 ? 1.0 : (nf >= 1e-5 ? 1.0 / nf : 1e5);
    }
    *dsig = sigma;
    s->cur ^= 1;
    s->f = ft;
    s->hist[s->len & 31] = ft;
    s->len += 1;
    s->k += 1;
    // the checks at the top of the next iteration
    if (!isfinite(s->f)) {
      s->bad = 1;
      s->done = 1;
    } else if (sqrt(s->f) <= s->tol_abs + s->tol_rel * s->nF0) {
      s->conv = 1;
      s->done = 1;
    } else {
      if (s->len > kDfsStag) {
        s->best_old = fmin(s->best_old, s->hist[(s->len - 1 - kDfsStag) & 31]);
        double best_new = INFINITY;
        for (int j = s->len - kDfsStag; j < s->len; ++j) best_new = fmin(best_new, s->hist[j & 31]);
        if (best_new > 0.81 * s->best_old) s->done = 1;
      }
      if (s->k >= s->max_iter) s->done = 1;
      if (!s->done) {
        double fm = 0;
        for (int j = s->len > kDfsM ? s->len - kDfsM : 0; j < s->len; ++j) fm = fmax(fm, s->hist[j & 31]);
        s->fmax = fm;
        s->eta = s->nF0 / ((1.0 + s->k) * (1.0 + s->k));
        s->ap = 1;
        s->am = 1;
        s->bt = 0;
        s->phase = 0;
      }
    }
  }
  if (s->trials >= s->max_trials) s->done = 1;
  cudaGraphSetConditional(cond, s->done ? 0u : 1u);
}

static bool device_dfsane_enabled() {
  static const bool on = [] {
    const char* e = getenv("FVIM_DEVICE_DFSANE");
    return !(e && e[0] == '0');
  }();
  return on;
}

inline DFS* dfs_dev(fvim_ctx* c) { return static_cast<DFS*>(c->sv[V_DFS]); }
inline double* dfs_sigma(fvim_ctx* c) { return reinterpret_cast<double*>(static_cast<char*>(c->sv[V_PKS]) + 128); }
inline unsigned* dfs_count(fvim_ctx* c) { return reinterpret_cast<unsigned*>(static_cast<char*>(c->sv[V_PKS]) + 196); }

// The WHILE graph of the device DF-SANE loop (built once per context; the material constants
// and the buffers are fixed, the points and the scalars live in the device state).
template <typename T> int build_dfloop(fvim_ctx* c, SolverRT* r, size_t n, int grd, int lgxy) {
  DFS* dfs = dfs_dev(c);
  return build_while_graph(
      c,
      [&](cudaGraphConditionalHandle cond) -> int {
        int e;
        if ((e = reset_flow_range(c))) return e;
        const size_t nv = n / 6;
        k_dfd_trial_rmap<T><<<(unsigned)((nv + 255) / 256), 256, 0, c->stream>>>(
            dfs, dfs_sigma(c), (const T*)c->st_sig, (const T*)c->st_ep, S<T>(c, V_DEP), (T*)nullptr,
            (size_t)c->n1 * c->n2, nv, (T)c->lam, (T)c->mu, (T)c->sigma_y, (T)c->E_h, flow_range(c));
        FVIM_CUDA_CHECK_LAUNCH();
        if ((e = apply_mindlin_t<T>(c, S<T>(c, V_DEP), S<T>(c, V_TMP), FVIM_STRAIN, nullptr, flow_range(c)))) return e;
        k_dfd_res_sy<T><<<grd, RT, 0, c->stream>>>(dfs, dfs_sigma(c), S<T>(c, V_B), S<T>(c, V_TMP),
                                                   (const double*)c->sv[V_WZ], lgxy, n, (double*)c->sv[V_PART],
                                                   dfs_count(c));
        k_dfd_decide<<<1, 32, 0, c->stream>>>(dfs, dfs_sigma(c), cond);
        FVIM_CUDA_CHECK_LAUNCH();
        return FVIM_OK;
      },
      &r->dfloop);
}

template <typename T>
int plasticity_t(fvim_ctx* c, const T* dT, T* dE, T* deps_p, T* dep, const fvim_opts* o, int* iters, double* res,
                 long* evals_out, bool warm = false) {
  const size_t nxy = (size_t)c->n1 * c->n2, n = nxy * c->nz * 6;
  int lgxy = 0;
  while (((size_t)1 << lgxy) < nxy) ++lgxy;
  DF<T> df{c, n, nxy, rgrid(sizeof(T) == 4 ? n / 4 : n), lgxy};
  int rc;
  // elastic predictor b = grad^sym M[dT], start x0 = b
  if ((rc = apply_boussinesq_t<T>(c, dT, nullptr, S<T>(c, V_B), FVIM_STRAIN))) return rc;
  T* x = S<T>(c, V_X);
  T* F = S<T>(c, V_F);
  T* xt = S<T>(c, V_XT);
  T* Ft = S<T>(c, V_FT);
  if (FVIM_CU(cudaMemcpyAsync(x, S<T>(c, V_B), n * sizeof(T), cudaMemcpyDeviceToDevice, c->stream)))
    return FVIM_ERR_CUDA;
  double f;
  if ((rc = df.eval(x, F, &f))) return rc;
  long evals = 1;
  // the stopping scale is the residual at the elastic predictor in every case
  const double nF0 = sqrt(f);
  if (warm) {
    // start from dE (the previous coupling iterate) when its residual is the smaller one
    double fw;
    if ((rc = df.eval(dE, Ft, &fw))) return rc;
    ++evals;
    if (fw < f) {
      if (FVIM_CU(cudaMemcpyAsync(x, dE, n * sizeof(T), cudaMemcpyDeviceToDevice, c->stream)))
        return FVIM_ERR_CUDA;
      std::swap(F, Ft);
      c->sv[V_F] = F;
      c->sv[V_FT] = Ft;
      f = fw;
    }
  }
  const int M = 10;
  const double gamma = 1e-4, smin = 1e-10, smax = 1e10, tmin = 0.1, tmax = 0.5;
  std::vector<double> hist(1, f);
  // the spectral step lives on the device (after the plasticity state block)
  double* dsig = reinterpret_cast<double*>(static_cast<char*>(c->sv[V_PKS]) + 128);
  k_set_double<<<1, 1, 0, c->stream>>>(dsig, 1.0);
  FVIM_CUDA_CHECK_LAUNCH();
  int k = 0;
  bool conv_ok = false;
  // stagnation at the rounding floor of the path precision: the best residual of the
  // last kStag iterations is not 10 % below the best one before them
  const int kStag = 30;
  double best_old = INFINITY;
  SolverRT* srt = rt(c);
  bool device_loop = srt && !c->prof && graphs_enabled() && device_dfsane_enabled() && o->df_max_iter > 0 &&
                     isfinite(f) && !(sqrt(f) <= o->df_tol_abs + o->df_tol_rel * nF0);
  if (device_loop && !srt->dfloop && !srt->dfloop_failed) {
    if (build_dfloop<T>(c, srt, n, df.grd, df.lgxy) != FVIM_OK) {
      srt->dfloop_failed = true;  // the host loop below takes over
      cudaGetLastError();
    }
  }
  bool ran_device = false;
  if (device_loop && srt->dfloop) {
    ran_device = true;
    DFS* hs = reinterpret_cast<DFS*>(reinterpret_cast<char*>(c->h_part) + (size_t)RMAXB * NVMAX * sizeof(double) + 256);
    memset(hs, 0, sizeof(DFS));
    hs->px[0] = x;
    hs->px[1] = xt;
    hs->pF[0] = F;
    hs->pF[1] = Ft;
    hs->f = f;
    hs->nF0 = nF0;
    hs->fmax = f;
    hs->eta = nF0;
    hs->ap = hs->am = 1.0;
    hs->best_old = INFINITY;
    hs->tol_abs = o->df_tol_abs;
    hs->tol_rel = o->df_tol_rel;
    hs->gamma = gamma;
    hs->smin = smin;
    hs->smax = smax;
    hs->tmin = tmin;
    hs->tmax = tmax;
    hs->hist[0] = f;
    hs->len = 1;
    hs->max_iter = o->df_max_iter;
    hs->max_trials = o->df_max_iter * 121 + 1;
    DFS* ds = dfs_dev(c);
    if (FVIM_CU(cudaMemcpyAsync(ds, hs, sizeof(DFS), cudaMemcpyHostToDevice, c->stream)) ||
        FVIM_CU(cudaMemsetAsync(dfs_count(c), 0, sizeof(unsigned), c->stream)) ||
        FVIM_CU(cudaGraphLaunch(srt->dfloop, c->stream)) ||
        FVIM_CU(cudaMemcpyAsync(hs, ds, sizeof(DFS), cudaMemcpyDeviceToHost, c->stream)) ||
        FVIM_CU(cudaStreamSynchronize(c->stream)))
      return FVIM_ERR_CUDA;
    c->n_applies += hs->evals;
    evals += hs->evals;
    k = hs->k;
    f = hs->f;
    conv_ok = hs->conv != 0;
    if (hs->bad) return FVIM_ERR_NONFINITE;
    x = const_cast<T*>(static_cast<const T*>(hs->px[hs->cur]));
    xt = const_cast<T*>(static_cast<const T*>(hs->px[1 - hs->cur]));
    F = static_cast<T*>(hs->pF[hs->cur]);
    Ft = static_cast<T*>(hs->pF[1 - hs->cur]);
    c->sv[V_X] = x;
    c->sv[V_XT] = xt;
    c->sv[V_F] = F;
    c->sv[V_FT] = Ft;
  }
  for (k = ran_device ? k : 0; !ran_device && k < o->df_max_iter; ++k) {
    if (!isfinite(f)) return FVIM_ERR_NONFINITE;
    if (sqrt(f) <= o->df_tol_abs + o->df_tol_rel * nF0) { conv_ok = true; break; }
    if (hist.size() > (size_t)kStag) {
      best_old = std::min(best_old, hist[hist.size() - 1 - kStag]);
      double best_new = INFINITY;
      for (size_t j = hist.size() - kStag; j < hist.size(); ++j) best_new = std::min(best_new, hist[j]);
      if (best_new > 0.81 * best_old) break;
    }
    double fmax = 0;
    for (size_t j = hist.size() > (size_t)M ? hist.size() - M : 0; j < hist.size(); ++j) fmax = std::max(fmax, hist[j]);
    const double eta = nF0 / ((1.0 + k) * (1.0 + k));
    double ap = 1, am = 1, fn = 0;
    bool ok = false;
    for (int bt = 0; bt < 60 && !ok; ++bt) {
      double fp, fm;
      // x + ap d with d = -sigma F
      if ((rc = axpby_vol<T>(c, xt, x, -ap, dsig, F, n))) return rc;
      if ((rc = df.eval(xt, Ft, &fp))) return rc;
      ++evals;
      if (fp <= fmax + eta - gamma * ap * ap * f) { fn = fp; ok = true; break; }
      if ((rc = axpby_vol<T>(c, xt, x, am, dsig, F, n))) return rc;
      if ((rc = df.eval(xt, Ft, &fm))) return rc;
      ++evals;
      if (fm <= fmax + eta - gamma * am * am * f) { fn = fm; ok = true; break; }
      ap = std::min(std::max(ap * ap * f / (fp + (2 * ap - 1) * f), tmin * ap), tmax * ap);
      am = std::min(std::max(am * am * f / (fm + (2 * am - 1) * f), tmin * am), tmax * am);
    }
    if (!ok) break;
    k_df_sy<T><<<df.grd, RT, 0, c->stream>>>(x, xt, F, Ft, (const double*)c->sv[V_WZ], df.lgxy, n,
                                             (double*)c->sv[V_PART]);
    k_df_sigma<<<1, RT, 0, c->stream>>>((const double*)c->sv[V_PART], df.grd, fn, smin, smax, dsig);
    FVIM_CUDA_CHECK_LAUNCH();
    std::swap(x, xt);
    std::swap(F, Ft);
    c->sv[V_X] = x;
    c->sv[V_XT] = xt;
    c->sv[V_F] = F;
    c->sv[V_FT] = Ft;
    f = fn;
    hist.push_back(f);
  }
  if (!conv_ok && sqrt(f) <= o->df_tol_abs + o->df_tol_rel * nF0) conv_ok = true;
  // outputs: dE = x and its return map
  if (FVIM_CU(cudaMemcpyAsync(dE, x, n * sizeof(T), cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
  if (deps_p || dep) {
    if ((rc = reset_flow_range(c))) return rc;
    if ((rc = return_map_t<T>(c, x, deps_p ? deps_p : S<T>(c, V_DEP), dep ? dep : S<T>(c, V_EP), flow_range(c))))
      return rc;
  }
  if (iters) *iters = k;
  if (res) *res = sqrt(f);
  if (evals_out) *evals_out += evals;
  return conv_ok ? FVIM_OK : FVIM_ERR_NOT_CONVERGED;
}

// ---- Algorithm 1 ---------------------------------------------------------------------
template <typename T>
int solve_contact_t(fvim_ctx* c, const T* h, const double* loads, int n_inc, const fvim_opts* o, T* p_out,
                    fvim_report* rep) {
  const size_t ns = (size_t)c->n1 * c->n2, nxy = ns, nv = nxy * c->nz;
  const double dA = c->L1 * c->L2 / (double)ns;
  int rc;
  T *H0 = S<T>(c, S_H0), *H = S<T>(c, S_H), *dU = S<T>(c, S_DU), *dUp = S<T>(c, S_DUPREV);
  T *P = S<T>(c, S_P), *Tprev = S<T>(c, S_TPREV), *dT = S<T>(c, S_DT);
  T* dE = S<T>(c, V_DE);
  const int gs = rgrid(ns);
  double v[2];
  int status = FVIM_OK;
  for (int inc = 0; inc < n_inc; ++inc) {
    const double W = loads[inc];
    // H0 = h - N[C:eps_p_n].e3 at z = 0 (Rem. modified_contact)
    if ((rc = apply_mindlin_t<T>(c, (const T*)c->st_eps_p, S<T>(c, V_TMP), FVIM_STRAIN, dU))) return rc;
    c->n_applies++;
    if ((rc = axpby<T>(c, H0, h, -1.0, dU, ns))) return rc;
    if ((rc = sum2<T>(c, H0, ns, v))) return rc;
    const double hnorm = sqrt(v[1]);
    if (FVIM_CU(cudaMemcpyAsync(H, H0, ns * sizeof(T), cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
    if (FVIM_CU(cudaMemsetAsync(dUp, 0, ns * sizeof(T), c->stream))) return FVIM_ERR_CUDA;
    if (FVIM_CU(cudaMemsetAsync(P, 0, ns * sizeof(T), c->stream))) return FVIM_ERR_CUDA;   // first guess: uniform
    // T_prev = pressure of the last converged increment
    if (FVIM_CU(cudaMemcpyAsync(Tprev, c->st_T, ns * sizeof(T), cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
    double e = INFINITY;
    int k = 1;
    while (true) {
      int cgi = 0, dfi = 0;
      rc = elastic_contact_t<T>(c, H, W, P, o, &cgi, nullptr);
      if (rep) rep->cg_iters += cgi;
      if (rc && rc != FVIM_ERR_NOT_CONVERGED) return rc;
      if ((rc = axpby<T>(c, dT, P, -1.0, Tprev, ns))) return rc;
      long ev = 0;
      // inside an increment DF-SANE starts from the previous iterate's dE (k > 1)
      rc = plasticity_t<T>(c, dT, dE, S<T>(c, V_DEP), S<T>(c, V_EP), o, &dfi, nullptr, &ev, k > 1);
      if (rep) { rep->df_iters += dfi; rep->residual_evals += ev; }
      if (rc && rc != FVIM_ERR_NOT_CONVERGED) return rc;
      // dU = N[C:deps_p].e3 at z = 0
      // V_DEP is the increment of the last return map, whose flow range is current
      if ((rc = apply_mindlin_t<T>(c, S<T>(c, V_DEP), S<T>(c, V_TMP), FVIM_STRAIN, dU, flow_range(c)))) return rc;
      c->n_applies++;
      k_diff2<T><<<gs, RT, 0, c->stream>>>(dU, dUp, ns, (double*)c->sv[V_PART]);
      FVIM_CUDA_CHECK_LAUNCH();
      if ((rc = finish<1>(c, gs, v))) return rc;
      e = sqrt(v[0]) / hnorm;
      // relaxation, modified surface, then dU_prev <- dU (Algorithm 1, literal order) or <- the
      // relaxed value (relax_mode FVIM_RELAX_CARRIED)
      k_relax<T><<<gs, RT, 0, c->stream>>>(H, H0, dUp, dU, o->relax, o->relax_mode == FVIM_RELAX_CARRIED ? 1 : 0,
                                           ns);
      FVIM_CUDA_CHECK_LAUNCH();
      k += 1;
      if (e < o->tol || k > o->max_iter) break;
    }
    // update(S, dE) and the converged pressure
    if ((rc = commit_t<T>(c, dE, S<T>(c, V_DEP), S<T>(c, V_EP)))) return rc;
    if (FVIM_CU(cudaMemcpyAsync(c->st_T, P, ns * sizeof(T), cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
    if ((rc = sum2<T>(c, P, ns, v))) return rc;
    double area[1];
    k_count_pos<T><<<gs, RT, 0, c->stream>>>(P, ns, (double*)c->sv[V_PART]);
    FVIM_CUDA_CHECK_LAUNCH();
    if ((rc = finish<1>(c, gs, area))) return rc;
    if (rep) {
      if (inc < FVIM_MAX_INCREMENTS) rep->contact_area[inc] = area[0] / (double)ns;
      rep->n_increments = inc + 1;
      if (inc < FVIM_MAX_INCREMENTS) {
        rep->alg1_iters[inc] = k - 1;
        rep->alg1_error[inc] = e;
      }
      rep->load_error = std::max(rep->load_error, fabs(dA * v[0] - W) / W);
    }
    if (!(e < o->tol)) status = FVIM_ERR_NOT_CONVERGED;
  }
  (void)nv;
  if (p_out && FVIM_CU(cudaMemcpyAsync(p_out, P, ns * sizeof(T), cudaMemcpyDeviceToDevice, c->stream))) return FVIM_ERR_CUDA;
  if (FVIM_CU(cudaStreamSynchronize(c->stream))) return FVIM_ERR_CUDA;
  return status;
}

}  // namespace

void solver_drop_graphs(fvim_ctx* c) {
  SolverRT* r = (SolverRT*)c->srt;
  if (!r) return;
  drop(r->cg);
  drop(r->df);
  drop(r->cgw);
  if (r->dfloop) cudaGraphExecDestroy(r->dfloop);
  r->dfloop = nullptr;
}

void solver_release(fvim_ctx* c) {
  SolverRT* r = (SolverRT*)c->srt;
  if (r) {
    drop(r->cg);
    drop(r->df);
    if (r->dfloop) cudaGraphExecDestroy(r->dfloop);
    if (r->stream) cudaStreamDestroy(r->stream);
    if (r->ev_in) cudaEventDestroy(r->ev_in);
    if (r->ev_out) cudaEventDestroy(r->ev_out);
    delete r;
    c->srt = nullptr;
  }
  if (c->h_part) cudaFreeHost(c->h_part);
  c->h_part = nullptr;
}

extern "C" {

int fvim_default_opts(const fvim_ctx* c, fvim_opts* o) {
  if (!c || !o) return FVIM_ERR_ARG;
  const bool dbl = c->prec == FVIM_FP64;
  o->tol = dbl ? 1e-9 : 1e-8;
  o->max_iter = 100;
  o->relax = 1.0;
  o->cg_tol = dbl ? 1e-12 : 1e-7;
  o->cg_max_iter = 2000;
  o->df_tol_abs = 0.0;
  o->df_tol_rel = dbl ? 1e-10 : 1e-6;
  o->df_max_iter = 500;
  o->relax_mode = FVIM_RELAX_LITERAL;
  return FVIM_OK;
}

static int check_opts(const fvim_opts* o) {
  if (!o) return FVIM_ERR_ARG;
  if (!(o->tol > 0) || o->max_iter < 1 || !(o->relax > 0 && o->relax <= 1) || !(o->cg_tol > 0) ||
      o->cg_max_iter < 1 || !(o->df_tol_abs >= 0) || !(o->df_tol_rel >= 0) || o->df_max_iter < 0 ||
      (o->relax_mode != FVIM_RELAX_LITERAL && o->relax_mode != FVIM_RELAX_CARRIED))
    return FVIM_ERR_ARG;
  return FVIM_OK;
}

int fvim_elastic_contact(fvim_ctx* c, const void* h, double W, void* p, const fvim_opts* o, int* iters, double* err) {
  if (!c || !h || !p || !(W > 0) || check_opts(o)) return FVIM_ERR_ARG;
  int rc = c->prec == FVIM_FP64 ? ensure_ws<double>(c) : ensure_ws<float>(c);
  if (rc) return rc;
  OnSolverStream on(c);
  if (c->prec == FVIM_FP64) return elastic_contact_t<double>(c, (const double*)h, W, (double*)p, o, iters, err);
  return elastic_contact_t<float>(c, (const float*)h, W, (float*)p, o, iters, err);
}

int fvim_plasticity_solve(fvim_ctx* c, const void* dT, void* dE, void* deps_p, void* dep, const fvim_opts* o,
                          int* iters, double* res) {
  if (!c || !dT || !dE || check_opts(o) || !isfinite(c->sigma_y)) return FVIM_ERR_ARG;
  int rc = c->prec == FVIM_FP64 ? ensure_ws<double>(c) : ensure_ws<float>(c);
  if (rc) return rc;
  OnSolverStream on(c);
  if (c->prec == FVIM_FP64)
    rc = plasticity_t<double>(c, (const double*)dT, (double*)dE, (double*)deps_p, (double*)dep, o, iters, res, nullptr);
  else
    rc = plasticity_t<float>(c, (const float*)dT, (float*)dE, (float*)deps_p, (float*)dep, o, iters, res, nullptr);
  if (FVIM_CU(cudaStreamSynchronize(c->stream))) return FVIM_ERR_CUDA;
  return rc;
}

int fvim_solve_contact(fvim_ctx* c, const void* h, const double* loads, int n_inc, const fvim_opts* o, void* p_out,
                       fvim_report* rep) {
  if (!c || !h || !loads || n_inc < 1 || check_opts(o) || !isfinite(c->sigma_y)) return FVIM_ERR_ARG;
  for (int i = 0; i < n_inc; ++i)
    if (!(loads[i] > 0) || !isfinite(loads[i])) return FVIM_ERR_ARG;
  if (rep) memset(rep, 0, sizeof(*rep));
  const long a0 = c->n_applies;
  int rc = c->prec == FVIM_FP64 ? ensure_ws<double>(c) : ensure_ws<float>(c);
  if (rc) return rc;
  {
    OnSolverStream on(c);
    if (c->prec == FVIM_FP64)
      rc = solve_contact_t<double>(c, (const double*)h, loads, n_inc, o, (double*)p_out, rep);
    else
      rc = solve_contact_t<float>(c, (const float*)h, loads, n_inc, o, (float*)p_out, rep);
  }
  if (rep) {
    rep->status = rc;
    rep->mindlin_applies = c->n_applies - a0;
  }
  return rc;
}

}  // extern "C"
