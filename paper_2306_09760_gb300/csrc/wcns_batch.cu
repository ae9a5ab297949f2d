// Batched 1D Euler problems: per-problem CFL steps, persistent stage kernels over a
// size-sorted (problem, tile) work list, one captured CUDA graph per RK3 step, and an
// autotuner that picks the tile (cells per work item) and resident blocks per SM by
// timing the candidates on the caller's data.  See include/wcns.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/wcns.h"
#include "wcns_batch_kernels.cuh"

using namespace wcns;

struct wcns_batch {
  int nprob;
  int64_t total;
  double lo, hi;
  int bc;
  int dtype;
  wcns_params p;
  Scheme s;
  cudaStream_t stream;
  int num_sms;
  std::vector<int64_t> h_off;
  std::vector<int> h_n;
  // device arrays
  int64_t* d_off;
  int* d_n;
  double* d_h;
  double* d_invh;
  StepDt* d_dt;       // per problem
  StepDt* d_tune_dt;
  double* d_t;
  long long* d_steps;
  unsigned int* d_tickets;   // [4]
  int* d_err;
  unsigned long long* d_fallbacks;
  BatchItem* d_items;
  int nitems;
  void* u1;
  void* u2;
  // launch configuration
  int nt;                     // threads per block (tile = nt - 5)
  int bps;                    // resident blocks per SM
  int candidates;
  bool configured;
  cudaGraphExec_t graph;
  const void* graph_u;
  double graph_tend;
};

namespace {

wcns_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return WCNS_OK;
  if (e == cudaErrorMemoryAllocation) return WCNS_ERR_NOMEM;
  return WCNS_ERR_CUDA;
}

#define WCNS_TRY(expr)                           \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return from_cuda(e_); \
  } while (0)


Scheme batch_scheme(const wcns_params* p) {
  Scheme s{};
  s.system = p->system;
  s.weights = p->weights;
  s.flux = p->flux;
  s.characteristic = p->characteristic ? 1 : 0;
  s.zp = p->z_p;
  s.renorm = p->renorm ? 1 : 0;
  s.gamma = p->gamma;
  s.eps = p->eps;
  s.xi = p->xi;
  s.cv = p->cv;
  s.harten = p->harten;
  s.speed[0] = p->alpha[0];
  s.speed[1] = p->alpha[1];
  fill_family_tables(s, p->family, p->kappa);
  return s;
}

// Work list for tiles of (nt - 5) cells, problems in decreasing size.
cudaError_t build_items(wcns_batch* b, int nt) {
  const int tile = nt - 5;
  std::vector<int> order(b->nprob);
  for (int k = 0; k < b->nprob; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->h_n[x] > b->h_n[y]; });
  std::vector<BatchItem> items;
  for (int k : order)
    for (int c0 = 0; c0 < b->h_n[k]; c0 += tile) items.push_back(BatchItem{k, c0});
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  cudaError_t e = cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
  b->nitems = (int)items.size();
  return e;
}

template <typename T, int NT, int FIX>
cudaError_t stage_launch(wcns_batch* b, const void* u, const void* un, void* out, double a, double c, int ticket,
                         const StepDt* dt, int bps) {
  BatchStageArgs<T> A{};
  A.u = static_cast<const T*>(u);
  A.un = static_cast<const T*>(un);
  A.out = static_cast<T*>(out);
  A.off = b->d_off;
  A.n = b->d_n;
  A.inv_h = b->d_invh;
  A.dt = dt;
  A.items = b->d_items;
  A.nitems = b->nitems;
  A.ticket = b->d_tickets + ticket;
  A.total = b->total;
  A.bc = b->bc;
  A.a = T(a);
  A.b = T(c);
  A.s = scheme_as<T>(b->s);
  A.fallbacks = b->d_fallbacks;
  batch_stage_kernel<T, NT, FIX><<<b->num_sms * bps, NT, 0, b->stream>>>(A);
  return cudaGetLastError();
}

bool batch_fixed(const Scheme& s) { return fixed_config(s); }

template <typename T, int FIX>
cudaError_t stage_fix(wcns_batch* b, int nt, const void* u, const void* un, void* out, double a, double c, int ticket,
                      const StepDt* dt, int bps) {
  switch (nt) {
    case 128: return stage_launch<T, 128, FIX>(b, u, un, out, a, c, ticket, dt, bps);
    case 256: return stage_launch<T, 256, FIX>(b, u, un, out, a, c, ticket, dt, bps);
    case 512: return stage_launch<T, 512, FIX>(b, u, un, out, a, c, ticket, dt, bps);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t stage_any(wcns_batch* b, int nt, const void* u, const void* un, void* out, double a, double c, int ticket,
                      const StepDt* dt, int bps) {
  return batch_fixed(b->s) ? stage_fix<T, 1>(b, nt, u, un, out, a, c, ticket, dt, bps)
                           : stage_fix<T, 0>(b, nt, u, un, out, a, c, ticket, dt, bps);
}

cudaError_t stage(wcns_batch* b, const void* u, const void* un, void* out, double a, double c, int ticket,
                  const StepDt* dt, int nt, int bps) {
  return b->dtype == WCNS_F64 ? stage_any<double>(b, nt, u, un, out, a, c, ticket, dt, bps)
                              : stage_any<float>(b, nt, u, un, out, a, c, ticket, dt, bps);
}

template <typename T, int FIX>
int max_blocks_fix(int nt) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (nt) {
    case 128: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_stage_kernel<T, 128, FIX>, 128, 0); break;
    case 256: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_stage_kernel<T, 256, FIX>, 256, 0); break;
    case 512: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_stage_kernel<T, 512, FIX>, 512, 0); break;
  }
  return e == cudaSuccess ? n : 0;
}

int max_blocks_per_sm(const wcns_batch* b, int nt) {
  const bool f = batch_fixed(b->s);
  if (b->dtype == WCNS_F64) return f ? max_blocks_fix<double, 1>(nt) : max_blocks_fix<double, 0>(nt);
  return f ? max_blocks_fix<float, 1>(nt) : max_blocks_fix<float, 0>(nt);
}

cudaError_t dt_launch(wcns_batch* b, const void* u, double t_end, StepDt* dt_out, int advance) {
  BatchDtArgs A{};
  A.u = u;
  A.off = b->d_off;
  A.n = b->d_n;
  A.h = b->d_h;
  A.dt = dt_out;
  A.t = b->d_t;
  A.steps = b->d_steps;
  A.total = b->total;
  A.gamma = b->p.gamma;
  A.cfl = b->p.cfl;
  A.t_end = t_end;
  A.advance = advance;
  A.err = b->d_err;
  if (b->dtype == WCNS_F64) batch_dt_kernel<double><<<b->nprob, 256, 0, b->stream>>>(A);
  else batch_dt_kernel<float><<<b->nprob, 256, 0, b->stream>>>(A);
  return cudaGetLastError();
}

cudaError_t rk3_step(wcns_batch* b, void* u, double t_end) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(b->d_tickets, 0, 4 * sizeof(unsigned int), b->stream)) != cudaSuccess) return e;
  if ((e = dt_launch(b, u, t_end, b->d_dt, 1)) != cudaSuccess) return e;
  if ((e = stage(b, u, nullptr, b->u1, 0.0, 1.0, 0, b->d_dt, b->nt, b->bps)) != cudaSuccess) return e;
  if ((e = stage(b, b->u1, u, b->u2, 0.75, 0.25, 1, b->d_dt, b->nt, b->bps)) != cudaSuccess) return e;
  return stage(b, b->u2, u, u, 1.0 / 3.0, 2.0 / 3.0, 2, b->d_dt, b->nt, b->bps);
}

// Times each (tile, blocks per SM) candidate on stage 1 of the caller's data (u is only
// read; u1 is scratch) and keeps the fastest.
cudaError_t autotune(wcns_batch* b, const void* u) {
  cudaError_t e;
  if ((e = dt_launch(b, u, 0.0, b->d_tune_dt, 0)) != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) return e;
  float best = 1e30f;
  int best_nt = 256, best_bps = 1, count = 0;
  const int nts[3] = {128, 256, 512};
  for (int nt : nts) {
    if ((e = build_items(b, nt)) != cudaSuccess) break;
    int maxb = max_blocks_per_sm(b, nt);
    for (int bps = 1; bps <= maxb; bps *= 2) {
      float tmin = 1e30f;
      for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaMemsetAsync(b->d_tickets + 3, 0, sizeof(unsigned int), b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = stage(b, u, nullptr, b->u1, 0.0, 1.0, 3, b->d_tune_dt, nt, bps);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tmin = std::min(tmin, ms);
      }
      if (e != cudaSuccess) break;
      ++count;
      if (tmin < best) {
        best = tmin;
        best_nt = nt;
        best_bps = bps;
      }
      if (bps * 2 > maxb && bps != maxb) {
        // also try the occupancy limit itself
        int last = maxb;
        float tm = 1e30f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
          e = cudaMemsetAsync(b->d_tickets + 3, 0, sizeof(unsigned int), b->stream);
          if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
          if (e == cudaSuccess) e = stage(b, u, nullptr, b->u1, 0.0, 1.0, 3, b->d_tune_dt, nt, last);
          if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) tm = std::min(tm, ms);
        }
        ++count;
        if (e == cudaSuccess && tm < best) {
          best = tm;
          best_nt = nt;
          best_bps = last;
        }
      }
    }
    if (e != cudaSuccess) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  b->nt = best_nt;
  b->bps = best_bps;
  b->candidates = count;
  return build_items(b, best_nt);
}

void drop_graph(wcns_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_u = nullptr;
}

}  // namespace

extern "C" {

wcns_status wcns_batch_init(const int64_t* offsets, const int64_t* n, int32_t nprob, int64_t total, double lo,
                            double hi, int32_t bc, const wcns_params* params, int32_t dtype, int32_t tile,
                            void* stream, wcns_batch** out) {
  if (!out) return WCNS_ERR_ARG;
  *out = nullptr;
  if (!offsets || !n || !params || nprob < 1 || total < 1 || !(hi > lo)) return WCNS_ERR_ARG;
  if (bc != WCNS_BC_PERIODIC && bc != WCNS_BC_TRANSMISSIVE) return WCNS_ERR_ARG;
  if (dtype != WCNS_F64 && dtype != WCNS_F32) return WCNS_ERR_ARG;
  if (tile != 0 && tile != 123 && tile != 251 && tile != 507) return WCNS_ERR_ARG;
  if (params->system != WCNS_EULER || params->integrator != WCNS_RK3) return WCNS_ERR_UNSUPPORTED;
  if (params->weights < WCNS_W_JS || params->weights > WCNS_W_M || params->flux < WCNS_FLUX_LLF ||
      params->flux > WCNS_FLUX_LLF_FROZEN || (params->z_p != 1 && params->z_p != 2) || !(params->eps > 0.0) ||
      !(params->gamma > 1.0) || !(params->cfl > 0.0))
    return WCNS_ERR_ARG;
  if (dtype == WCNS_F32 && (params->weights == WCNS_W_JS || params->weights == WCNS_W_M) && params->eps < 1e-18)
    return WCNS_ERR_ARG;
  if (nprob > (1 << 30) || total > ((int64_t)1 << 34)) return WCNS_ERR_ARG;
  for (int32_t k = 0; k < nprob; ++k) {
    if (n[k] < 1 || n[k] > (1 << 30) || offsets[k] < 0 || offsets[k] + n[k] > total) return WCNS_ERR_ARG;
  }
  {  // problems must not overlap
    std::vector<std::pair<int64_t, int64_t>> iv(nprob);
    for (int32_t k = 0; k < nprob; ++k) iv[k] = {offsets[k], offsets[k] + n[k]};
    std::sort(iv.begin(), iv.end());
    for (int32_t k = 1; k < nprob; ++k)
      if (iv[k].first < iv[k - 1].second) return WCNS_ERR_ARG;
  }
  wcns_batch* b = new (std::nothrow) wcns_batch();
  if (!b) return WCNS_ERR_NOMEM;
  b->nprob = nprob;
  b->total = total;
  b->lo = lo;
  b->hi = hi;
  b->bc = bc;
  b->dtype = dtype;
  b->p = *params;
  b->s = batch_scheme(params);
  b->stream = static_cast<cudaStream_t>(stream);
  b->h_off.assign(offsets, offsets + nprob);
  b->h_n.resize(nprob);
  std::vector<double> h(nprob), ih(nprob);
  for (int k = 0; k < nprob; ++k) {
    b->h_n[k] = (int)n[k];
    h[k] = (hi - lo) / (double)n[k];
    ih[k] = 1.0 / h[k];
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t elem = dtype == WCNS_F64 ? 8 : 4;
  if (e == cudaSuccess) e = cudaMalloc(&b->d_off, sizeof(int64_t) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_n, sizeof(int) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_h, sizeof(double) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_invh, sizeof(double) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_dt, sizeof(StepDt) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tune_dt, sizeof(StepDt) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_t, sizeof(double) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_steps, sizeof(long long) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tickets, 64);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_err, 64);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_fallbacks, 64);
  if (e == cudaSuccess) e = cudaMalloc(&b->u1, elem * 3 * total);
  if (e == cudaSuccess) e = cudaMalloc(&b->u2, elem * 3 * total);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_off, offsets, sizeof(int64_t) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_n, b->h_n.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_h, h.data(), sizeof(double) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_invh, ih.data(), sizeof(double) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_t, 0, sizeof(double) * nprob);
  if (e == cudaSuccess) e = cudaMemset(b->d_steps, 0, sizeof(long long) * nprob);
  if (e == cudaSuccess) e = cudaMemset(b->d_tickets, 0, 64);
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, 64);
  if (e == cudaSuccess) e = cudaMemset(b->d_fallbacks, 0, 64);
  if (e == cudaSuccess && tile != 0) {
    b->nt = tile + 5;
    int maxb = max_blocks_per_sm(b, b->nt);
    b->bps = maxb > 0 ? maxb : 1;
    b->configured = true;
    e = build_items(b, b->nt);
  }
  if (e != cudaSuccess) {
    wcns_batch_destroy(b);
    return from_cuda(e);
  }
  *out = b;
  return WCNS_OK;
}

wcns_status wcns_batch_step(wcns_batch* b, void* u, int32_t nsteps, double t_end) {
  if (!b || !u || nsteps < 0 || t_end != t_end) return WCNS_ERR_ARG;
  if (nsteps == 0) return WCNS_OK;
  if (!b->configured) {
    WCNS_TRY(autotune(b, u));
    b->configured = true;
  }
  if (b->stream != nullptr) {
    if (!b->graph || b->graph_u != u || b->graph_tend != t_end) {
      drop_graph(b);
      cudaGraph_t g = nullptr;
      WCNS_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t body = rk3_step(b, u, t_end);
      cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      if (body != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return from_cuda(body != cudaSuccess ? body : e);
      }
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        return from_cuda(e);
      }
      b->graph_u = u;
      b->graph_tend = t_end;
    }
    for (int32_t k = 0; k < nsteps; ++k) WCNS_TRY(cudaGraphLaunch(b->graph, b->stream));
    return WCNS_OK;
  }
  for (int32_t k = 0; k < nsteps; ++k) WCNS_TRY(rk3_step(b, u, t_end));
  return WCNS_OK;
}

wcns_status wcns_batch_config(wcns_batch* b, int32_t* tile, int32_t* bps, int32_t* candidates) {
  if (!b) return WCNS_ERR_ARG;
  if (tile) *tile = b->configured ? b->nt - 5 : 0;
  if (bps) *bps = b->configured ? b->bps : 0;
  if (candidates) *candidates = b->candidates;
  return WCNS_OK;
}

wcns_status wcns_batch_times(wcns_batch* b, double* t_host) {
  if (!b || !t_host) return WCNS_ERR_ARG;
  WCNS_TRY(cudaMemcpyAsync(t_host, b->d_t, sizeof(double) * b->nprob, cudaMemcpyDeviceToHost, b->stream));
  WCNS_TRY(cudaStreamSynchronize(b->stream));
  return WCNS_OK;
}

wcns_status wcns_batch_sync_status(wcns_batch* b, int64_t* nonphysical) {
  if (!b) return WCNS_ERR_ARG;
  int err = 0;
  unsigned long long fb = 0;
  WCNS_TRY(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  WCNS_TRY(cudaMemcpyAsync(&fb, b->d_fallbacks, sizeof(fb), cudaMemcpyDeviceToHost, b->stream));
  WCNS_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
  WCNS_TRY(cudaMemsetAsync(b->d_fallbacks, 0, sizeof(fb), b->stream));
  WCNS_TRY(cudaStreamSynchronize(b->stream));
  if (nonphysical) *nonphysical = (int64_t)fb;
  if (err & 2) return WCNS_ERR_TIMEOUT;
  if (err & 1) return WCNS_ERR_NONPHYSICAL;
  return WCNS_OK;
}

void wcns_batch_destroy(wcns_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  void* ptrs[] = {b->d_off, b->d_n, b->d_h, b->d_invh, b->d_dt, b->d_tune_dt, b->d_t, b->d_steps,
                  b->d_tickets, b->d_err, b->d_fallbacks, b->d_items, b->u1, b->u2};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete b;
}

}  // extern "C"
