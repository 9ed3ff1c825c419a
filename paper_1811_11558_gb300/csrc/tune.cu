// Tile-plan autotuner of the depth kernel (declarations and contracts in include/fvim.h).
//
// The depth range of every mode is cut into chunks of C nodes, one thread per chunk, whose
// recursion carries are combined by a log-depth scan (depth.cu).  Short chunks give more
// threads and a shorter serial recursion, long chunks fewer scan rounds and fewer threads
// per tile; which one is fastest depends on the grid (small grids are latency bound, large
// ones issue bound), so it is measured: every launchable C is timed on the context's own
// stream and the fastest is kept in a process-wide table keyed by grid, precision and depth
// spacing, so later contexts of that grid start with it.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fvim_internal.cuh"

namespace {

typedef std::tuple<int, int, int, int, int> PlanKey;  // precision, n1, n2, nz, uniform

std::mutex g_plan_mu;
std::map<PlanKey, int>& plan_table() {
  static std::map<PlanKey, int> t;
  return t;
}

PlanKey key_of(const fvim_ctx* c) { return PlanKey(c->prec, c->n1, c->n2, c->nz, c->uniform); }

// candidate chunk lengths: the instantiated register-variant lengths, two longer ones, and
// the default rule
std::vector<int> candidates(const fvim_ctx* c) {
  std::vector<int> v;
  const int base[] = {2, 3, 4, 6, 8, 12, 16, depth_chunk_default(c->nz)};
  for (int C : base)
    if (depth_chunk_ok(c, C) && std::find(v.begin(), v.end(), C) == v.end()) v.push_back(C);
  if ((int)v.size() > FVIM_PLAN_MAX_CAND) v.resize(FVIM_PLAN_MAX_CAND);
  return v;
}

int launch_depth(const fvim_ctx* c) {
  return c->prec == FVIM_FP64 ? launch_mindlin_depth<double>(c, FVIM_STRESS, false)
                              : launch_mindlin_depth<float>(c, FVIM_STRESS, false);
}

// median of reps launch times of the depth kernel with chunk length C (ms), or < 0 on error
float time_chunk(fvim_ctx* c, int C, int reps, std::vector<cudaEvent_t>& ev) {
  c->depth_chunk = C;
  for (int w = 0; w < 2; ++w)
    if (launch_depth(c)) return -1.f;
  for (int r = 0; r < reps; ++r) {
    if (FVIM_CU(cudaEventRecord(ev[r], c->stream))) return -1.f;
    if (launch_depth(c)) return -1.f;
  }
  if (FVIM_CU(cudaEventRecord(ev[reps], c->stream))) return -1.f;
  if (FVIM_CU(cudaEventSynchronize(ev[reps]))) return -1.f;
  std::vector<float> t(reps);
  for (int r = 0; r < reps; ++r)
    if (FVIM_CU(cudaEventElapsedTime(&t[r], ev[r], ev[r + 1]))) return -1.f;
  std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
  return t[reps / 2];
}

void fill_plan(const fvim_ctx* c, fvim_plan* out) {
  out->depth_chunk = c->depth_chunk > 0 ? c->depth_chunk : depth_chunk_default(c->nz);
  out->tuned = c->plan_tuned;
}

}  // namespace

int plan_lookup(const fvim_ctx* c) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = plan_table().find(key_of(c));
  return it == plan_table().end() ? 0 : it->second;
}

extern "C" {

int fvim_autotune(fvim_ctx* c, int reps, fvim_plan* out) {
  if (!c || reps < 1 || reps > 1000) return FVIM_ERR_ARG;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (FVIM_CU(cudaStreamIsCapturing(c->stream, &cs))) return FVIM_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return FVIM_ERR_ARG;
  const std::vector<int> cand = candidates(c);
  if (cand.empty()) return FVIM_ERR_UNSUPPORTED;
  const int old = c->depth_chunk > 0 ? c->depth_chunk : depth_chunk_default(c->nz);
  // the kernel runs in place on the context's spectrum scratch; zeros take the same path
  const size_t es = c->prec == FVIM_FP64 ? 8 : 4;
  if (FVIM_CU(cudaMemsetAsync(c->spec, 0, (size_t)c->nz * 6 * c->n2 * c->h1 * 2 * es, c->stream))) return FVIM_ERR_CUDA;
  std::vector<cudaEvent_t> ev(reps + 1, nullptr);
  int rc = FVIM_OK;
  for (auto& e : ev)
    if (FVIM_CU(cudaEventCreate(&e))) { rc = FVIM_ERR_CUDA; break; }
  std::vector<float> ms(cand.size(), -1.f);
  for (size_t i = 0; rc == FVIM_OK && i < cand.size(); ++i) {
    ms[i] = time_chunk(c, cand[i], reps, ev);
    if (ms[i] < 0) rc = FVIM_ERR_CUDA;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (rc) {
    c->depth_chunk = old;
    return rc;
  }
  // the default rule keeps its place unless another length is faster by more than 2 %
  // (timing noise does not flip the plan)
  const int def = depth_chunk_default(c->nz);
  size_t best = 0;
  for (size_t i = 1; i < cand.size(); ++i)
    if (ms[i] < ms[best]) best = i;
  for (size_t i = 0; i < cand.size(); ++i)
    if (cand[i] == def && ms[best] > 0.98f * ms[i]) best = i;
  c->depth_chunk = cand[best];
  c->plan_tuned = 1;
  if (c->depth_chunk != old) solver_drop_graphs(c);  // captured graphs hold the old launch shape
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    plan_table()[key_of(c)] = c->depth_chunk;
  }
  if (out) {
    memset(out, 0, sizeof(*out));
    fill_plan(c, out);
    out->n_cand = (int)cand.size();
    for (size_t i = 0; i < cand.size(); ++i) {
      out->cand[i] = cand[i];
      out->cand_ms[i] = ms[i];
    }
  }
  return FVIM_OK;
}

int fvim_plan_candidates(int n1, int n2, int nz, int precision, int* chunks, int max_chunks) {
  if (!grid_ok(n1, n2) || nz < 2 || nz > 512) return FVIM_ERR_ARG;
  if ((precision != FVIM_FP32 && precision != FVIM_FP64) || !chunks || max_chunks < 1) return FVIM_ERR_ARG;
  // the launch rules need the grid and precision only: a host-side description of the grid
  fvim_ctx g;
  memset(&g, 0, sizeof(g));
  g.n1 = n1;
  g.n2 = n2;
  g.nz = nz;
  g.gen = grid_gen(n1, n2) ? 1 : 0;
  g.h1 = spec_stride(n1, n2);
  g.hs = g.gen ? n1 / 2 + 1 : g.h1;
  g.prec = precision;
  const std::vector<int> cand = candidates(&g);
  const int n = (int)cand.size() < max_chunks ? (int)cand.size() : max_chunks;
  for (int i = 0; i < n; ++i) chunks[i] = cand[i];
  return n;
}

int fvim_get_plan(const fvim_ctx* c, fvim_plan* out) {
  if (!c || !out) return FVIM_ERR_ARG;
  memset(out, 0, sizeof(*out));
  fill_plan(c, out);
  return FVIM_OK;
}

int fvim_set_plan(fvim_ctx* c, const fvim_plan* plan) {
  if (!c || !plan) return FVIM_ERR_ARG;
  const int C = plan->depth_chunk;
  if (C != 0 && !depth_chunk_ok(c, C)) return FVIM_ERR_ARG;
  const int old = c->depth_chunk > 0 ? c->depth_chunk : depth_chunk_default(c->nz);
  c->depth_chunk = C;
  c->plan_tuned = 0;
  if ((C > 0 ? C : depth_chunk_default(c->nz)) != old) solver_drop_graphs(c);
  return FVIM_OK;
}

}  // extern "C"
