// Batched scheduler: many independent reconstructions of uneven size side by
// side on one GPU.  Host C++ only; every kernel is the single-problem path's.
//
// A work queue in longest-first order feeds `lanes` workers.  Each worker owns a
// stream, a sub-handle (its own workspace and eigen-solver warm-start state) and
// a host thread that issues its problems' kernels, so the launch overhead of the
// small problems is spread over host cores and their kernels overlap on the GPU.
// Per-problem start and completion times come from events on the lanes' streams,
// measured from one event recorded on the caller's stream.
#include <algorithm>
#include <atomic>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "hicu_internal.cuh"

namespace hicu {

// Estimated floating-point operations of one problem: per outer iteration the lag-form
// Gram (8 C^2 (2k-1)^d flops per output position), about six warm Jacobi sweeps
// (48 n^2 flops per round, n - 1 rounds), and per descent step three convolutions of
// 8 n p flops per output position (conv, adjoint, the line-search conv).
static double problem_cost(const hicu_problem& P) {
  const hicu_geom& g = P.geom;
  if (g.ncoil < 1 || !P.params.stages || P.params.nstages < 1) return 0.0;
  const double C = g.ncoil;
  double lags = 1.0, K = 1.0;
  for (int a = 0; a < 3; ++a) {
    lags *= 2.0 * g.k[a] - 1.0;
    K *= g.k[a];
  }
  const double n = C * K;
  double cost = 0.0;
  for (int i = 0; i < P.params.nstages; ++i) {
    const hicu_stage& st = P.params.stages[i];
    double s = 1.0;
    for (int a = 0; a < 3; ++a) {
      const double e = (double)st.region.ext[a];
      s *= g.circular[a] ? e : std::max(0.0, e - g.k[a] + 1.0);
    }
    const double per_iter = 8.0 * C * C * lags * s + 6.0 * 48.0 * n * n * (n - 1.0) +
                            (double)st.gd_steps * 3.0 * 8.0 * n * (double)st.p * s;
    cost += (double)std::max(st.iters, 0) * per_iter;
  }
  return cost;
}

static int64_t problem_steps(const hicu_problem& P) {
  int64_t k = 0;
  for (int i = 0; P.params.stages && i < P.params.nstages; ++i)
    k += (int64_t)std::max(P.params.stages[i].iters, 0) * std::max(P.params.stages[i].gd_steps, 0);
  return k;
}

}  // namespace hicu

using namespace hicu;

extern "C" hicu_status hicu_batch_order(int32_t nslices, const hicu_problem* problems, int32_t* order,
                                        double* cost) {
  if (nslices < 0 || (nslices > 0 && (!problems || !order))) return HICU_ERR_ARG;
  std::vector<double> c(nslices);
  for (int i = 0; i < nslices; ++i) c[i] = problem_cost(problems[i]);
  std::vector<int32_t> idx(nslices);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return c[a] > c[b]; });
  for (int i = 0; i < nslices; ++i) {
    order[i] = idx[i];
    if (cost) cost[i] = c[i];
  }
  return HICU_OK;
}

extern "C" hicu_status hicu_reconstruct_batched(hicu_handle* h, int32_t nslices, const hicu_problem* problems,
                                                int32_t lanes, hicu_slice_report* report, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (nslices < 0 || (nslices > 0 && !problems)) return set_error(h, HICU_ERR_ARG, "batched: bad problem list");
  if (lanes < 0 || lanes > 64) return set_error(h, HICU_ERR_ARG, "batched: lanes must be in [0, 64]");
  if (nslices == 0) return HICU_OK;
  const int L = std::min<int>(lanes > 0 ? lanes : std::min(nslices, 8), nslices);
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_error(h, e, "batched: device");
  while ((int)h->lane_h.size() < L) {
    hicu_handle* c = nullptr;
    hicu_status s = hicu_create(&c);
    if (s) return set_error(h, s, "batched: lane handle");
    cudaStream_t ls = nullptr;
    e = cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      hicu_destroy(c);
      return cuda_error(h, e, "batched: lane stream");
    }
    h->lane_h.push_back(c);
    h->lane_st.push_back(ls);
  }
  if (!h->coop_st_own) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    e = cudaStreamCreateWithPriority(&h->coop_st_own, cudaStreamNonBlocking, hi);
    if (e != cudaSuccess) return cuda_error(h, e, "batched: priority stream");
  }
  for (int i = 0; i < L; ++i) {
    hicu_handle* c = h->lane_h[i];
    c->auto_cluster_max = 256;  // cluster solver wherever it applies
    c->coop_mu = &h->coop_mu_own;
    c->coop_st = h->coop_st_own;
    if (!c->coop_in && cudaEventCreateWithFlags(&c->coop_in, cudaEventDisableTiming) != cudaSuccess)
      return cuda_error(h, cudaGetLastError(), "batched: event");
    if (!c->coop_out && cudaEventCreateWithFlags(&c->coop_out, cudaEventDisableTiming) != cudaSuccess)
      return cuda_error(h, cudaGetLastError(), "batched: event");
  }
  while ((int)h->batch_ev.size() < 2 * nslices + 1) {
    cudaEvent_t ev;
    e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return cuda_error(h, e, "batched: events");
    h->batch_ev.push_back(ev);
  }
  cudaEvent_t t0 = h->batch_ev[0];
  std::vector<int32_t> order(nslices);
  hicu_batch_order(nslices, problems, order.data(), nullptr);

  cudaStream_t st = (cudaStream_t)stream;
  e = cudaEventRecord(t0, st);
  if (e != cudaSuccess) return cuda_error(h, e, "batched: start event");
  for (int i = 0; i < L; ++i) cudaStreamWaitEvent(h->lane_st[i], t0, 0);

  std::vector<long long> launches0(L);
  for (int i = 0; i < L; ++i) launches0[i] = h->lane_h[i]->launches_all;
  std::atomic<int> next(0);
  std::vector<int32_t> status(nslices, HICU_OK), lane_of(nslices, -1);
  std::vector<std::string> msg(nslices);
  auto worker = [&](int li) {
    cudaSetDevice(h->device);
    hicu_handle* c = h->lane_h[li];
    cudaStream_t ls = h->lane_st[li];
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= nslices) break;
      const int idx = order[k];
      const hicu_problem& P = problems[idx];
      cudaEventRecord(h->batch_ev[1 + 2 * idx], ls);
      const hicu_status s = hicu_reconstruct(c, &P.geom, P.x0, P.mask, &P.params, P.x_out, P.log, ls);
      cudaEventRecord(h->batch_ev[2 + 2 * idx], ls);
      status[idx] = s;
      lane_of[idx] = li;
      if (s) msg[idx] = c->last_error;
    }
  };
  std::vector<std::thread> threads;
  threads.reserve(L);
  for (int i = 0; i < L; ++i) threads.emplace_back(worker, i);
  for (auto& t : threads) t.join();

  // completion: a device-side error word on a lane (a bounded wait that gave up) is
  // charged to every problem that lane ran
  for (int i = 0; i < L; ++i) {
    hicu_handle* c = h->lane_h[i];
    const hicu_status s = hicu_check(c, h->lane_st[i]);
    if (s) {
      for (int idx = 0; idx < nslices; ++idx)
        if (lane_of[idx] == i && status[idx] == HICU_OK) {
          status[idx] = s;
          msg[idx] = c->last_error;
        }
    }
    h->launches_all += c->launches_all - launches0[i];
  }
  for (int idx = 0; idx < nslices && report; ++idx) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, t0, h->batch_ev[1 + 2 * idx]) != cudaSuccess ||
        cudaEventElapsedTime(&b, t0, h->batch_ev[2 + 2 * idx]) != cudaSuccess) {
      cudaGetLastError();
      a = b = -1.f;
    }
    report[idx].start_ms = a;
    report[idx].end_ms = b;
    report[idx].lane = lane_of[idx];
    report[idx].status = status[idx];
    report[idx].gd_steps = problem_steps(problems[idx]);
  }
  for (int idx = 0; idx < nslices; ++idx)
    if (status[idx] != HICU_OK)
      return set_error(h, (hicu_status)status[idx], "batched: problem " + std::to_string(idx) + ": " + msg[idx]);
  return HICU_OK;
}
