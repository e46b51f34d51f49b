// C ABI of libhicu: handle, argument validation, workspace, and the drivers
// that chain the kernels into the steps of Algorithm 1.
#include <cmath>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "hicu_internal.cuh"

namespace hicu {

hicu_status set_error(hicu_handle* h, hicu_status s, const std::string& msg) {
  if (h) h->last_error = msg;
  return s;
}

cudaError_t allow_max_dynamic_smem(const void* kernel) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, cudaError_t> done;
  // per host thread: the (kernel, device) pairs already raised, checked without the lock
  thread_local std::vector<std::pair<const void*, int>> seen;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  for (const auto& kd : seen)
    if (kd.first == kernel && kd.second == dev) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find({kernel, dev});
  if (it != done.end()) {
    if (it->second == cudaSuccess) seen.push_back({kernel, dev});
    return it->second;
  }
  int optin = 0;
  cudaFuncAttributes fa;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) cudaGetLastError();
  done[{kernel, dev}] = e;
  if (e == cudaSuccess) seen.push_back({kernel, dev});
  return e;
}

hicu_status cuda_error(hicu_handle* h, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return HICU_OK;
  return set_error(h, HICU_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

hicu_status ensure_side_stream(hicu_handle* h) {
  if (h->side_st) return HICU_OK;
  if (cudaStreamCreateWithFlags(&h->side_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->side_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->side_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->draw_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->draw_join, cudaEventDisableTiming) != cudaSuccess)
    return cuda_error(h, cudaGetLastError(), "side stream");
  return HICU_OK;
}

static hicu_status ensure_copy_stream(hicu_handle* h) {
  if (h->copy_st) return HICU_OK;
  if (cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->copy_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->copy_join, cudaEventDisableTiming) != cudaSuccess)
    return cuda_error(h, cudaGetLastError(), "copy stream");
  return HICU_OK;
}

void prof_count(hicu_handle* h, int cls) {
  ++h->launches_all;
  if (h->prof_class == cls) ++h->launches_class;
}

void prof_begin(hicu_handle* h, int cls, cudaStream_t st) {
  ++h->launches_all;
  if (h->prof_class != cls) return;
  ++h->launches_class;
  if (h->prof_used + 2 > (size_t)(1 << 16)) return;  // cap the number of timed launches
  while (h->prof_events.size() < h->prof_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    h->prof_events.push_back(e);
  }
  cudaEventRecord(h->prof_events[h->prof_used], st);
}

void prof_end(hicu_handle* h, int cls, cudaStream_t st) {
  if (h->prof_class != cls || h->prof_used + 2 > h->prof_events.size()) return;
  cudaEventRecord(h->prof_events[h->prof_used + 1], st);
  h->prof_used += 2;
}

void* ws_get(hicu_handle* h, int slot, size_t bytes, hicu_status* st) {
  Workspace& w = h->ws[slot];
  if (bytes == 0) bytes = 16;
  if (w.bytes >= bytes) return w.ptr;
  if (w.ptr) {
    cudaFree(w.ptr);  // synchronising; only happens while the workspace grows
    w.ptr = nullptr;
    w.bytes = 0;
  }
  void* p = nullptr;
  const size_t want = (bytes + 255) / 256 * 256;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    *st = set_error(h, HICU_ERR_ALLOC, "workspace allocation of " + std::to_string(want) + " bytes failed");
    return nullptr;
  }
  w.ptr = p;
  w.bytes = want;
  return p;
}

static bool geom_ok(const hicu_geom* g) {
  if (!g) return false;
  if (g->ncoil < 1 || g->ncoil > 64) return false;
  for (int a = 0; a < 3; ++a) {
    if (g->dim[a] < 1 || g->dim[a] > (1 << 20)) return false;
    if (g->k[a] < 1 || g->k[a] > 64) return false;
    if (g->circular[a] > 1) return false;
  }
  if (g->mask_per_coil > 1) return false;
  const long long N = g->dim[0] * g->dim[1] * g->dim[2] * (long long)g->ncoil;
  return N < (1ll << 40);
}

hicu_status make_conv_geom(hicu_handle* h, const hicu_geom* geom, const hicu_region* r,
                           ConvGeom* out) {
  if (!geom || !r) return set_error(h, HICU_ERR_ARG, "null geometry or region");
  if (!geom_ok(geom)) return set_error(h, HICU_ERR_SHAPE, "invalid geometry");
  ConvGeom g;
  g.C = geom->ncoil;
  g.kx = geom->k[0];
  g.ky = geom->k[1];
  g.kz = geom->k[2];
  g.K = g.kx * g.ky * g.kz;
  g.n = g.C * g.K;
  int ext[3], out_ext[3];
  for (int a = 0; a < 3; ++a) {
    if (r->off[a] < 0 || r->ext[a] < 1 || r->off[a] + r->ext[a] > geom->dim[a])
      return set_error(h, HICU_ERR_SHAPE, "region does not fit inside the array");
    ext[a] = (int)r->ext[a];
    if (geom->circular[a]) {
      out_ext[a] = ext[a];
    } else {
      if (ext[a] < geom->k[a]) return set_error(h, HICU_ERR_SHAPE, "region smaller than the kernel");
      out_ext[a] = ext[a] - geom->k[a] + 1;
    }
  }
  g.ex = ext[0];
  g.ey = ext[1];
  g.ez = ext[2];
  g.sx = out_ext[0];
  g.sy = out_ext[1];
  g.sz = out_ext[2];
  g.cx = geom->circular[0];
  g.cy = geom->circular[1];
  g.cz = geom->circular[2];
  g.s = (long long)g.sx * g.sy * g.sz;
  if (g.sy > 65535 * 4 || g.sz > 65535 || g.ez > 65535)
    return set_error(h, HICU_ERR_UNSUPPORTED, "region extent above launch limits");
  *out = g;
  return HICU_OK;
}

KView full_view(const hicu_geom* g, const hicu_region* r, float* base) {
  KView v;
  v.p = reinterpret_cast<float2*>(base);
  v.sy = g->dim[0];
  v.sz = g->dim[0] * g->dim[1];
  v.sc = v.sz * g->dim[2];
  v.ox = (int)r->off[0];
  v.oy = (int)r->off[1];
  v.oz = (int)r->off[2];
  return v;
}

static KView region_view(const ConvGeom& g, float2* base) {
  KView v;
  v.p = base;
  v.sy = g.ex;
  v.sz = (long long)g.ex * g.ey;
  v.sc = v.sz * g.ez;
  v.ox = v.oy = v.oz = 0;
  return v;
}

MView mask_view(const hicu_geom* g, const hicu_region* r, const uint8_t* mask) {
  MView m;
  m.p = mask;
  m.sy = g->dim[0];
  m.sz = g->dim[0] * g->dim[1];
  m.sc = g->mask_per_coil ? m.sz * g->dim[2] : 0;
  m.ox = (int)r->off[0];
  m.oy = (int)r->off[1];
  m.oz = (int)r->off[2];
  return m;
}

}  // namespace hicu

using namespace hicu;

// --------------------------------------------------------------- handle

extern "C" hicu_status hicu_create(hicu_handle** out) {
  if (!out) return HICU_ERR_ARG;
  *out = nullptr;
  hicu_handle* h = new (std::nothrow) hicu_handle();
  if (!h) return HICU_ERR_ALLOC;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return HICU_ERR_CUDA;
  }
  if (cudaMalloc(&h->dev_err, 64) != cudaSuccess || cudaMalloc(&h->dev_sync, 64) != cudaSuccess ||
      cudaMemset(h->dev_err, 0, 64) != cudaSuccess || cudaMemset(h->dev_sync, 0, 64) != cudaSuccess) {
    cudaGetLastError();
    if (h->dev_err) cudaFree(h->dev_err);
    if (h->dev_sync) cudaFree(h->dev_sync);
    delete h;
    return HICU_ERR_ALLOC;
  }
  const char* pdl_env = std::getenv("HICU_PDL");
  h->pdl = !(pdl_env && pdl_env[0] == '0');
  *out = h;
  return HICU_OK;
}

extern "C" hicu_status hicu_destroy(hicu_handle* h) {
  if (!h) return HICU_ERR_ARG;
  cudaDeviceSynchronize();
  for (auto* c : h->lane_h) hicu_destroy(c);
  for (auto st : h->lane_st) cudaStreamDestroy(st);
  for (auto e : h->batch_ev) cudaEventDestroy(e);
  if (h->coop_st_own) cudaStreamDestroy(h->coop_st_own);
  if (h->side_st) cudaStreamDestroy(h->side_st);
  if (h->side_fork) cudaEventDestroy(h->side_fork);
  if (h->side_join) cudaEventDestroy(h->side_join);
  if (h->draw_fork) cudaEventDestroy(h->draw_fork);
  if (h->draw_join) cudaEventDestroy(h->draw_join);
  if (h->copy_st) cudaStreamDestroy(h->copy_st);
  if (h->copy_fork) cudaEventDestroy(h->copy_fork);
  if (h->copy_join) cudaEventDestroy(h->copy_join);
  if (h->coop_in) cudaEventDestroy(h->coop_in);
  if (h->coop_out) cudaEventDestroy(h->coop_out);
  for (auto& w : h->ws)
    if (w.ptr) cudaFree(w.ptr);
  for (auto e : h->prof_events) cudaEventDestroy(e);
  release_fft(h);
  cudaFree(h->dev_err);
  cudaFree(h->dev_sync);
  delete h;
  return HICU_OK;
}

extern "C" const char* hicu_last_error(const hicu_handle* h) { return h ? h->last_error.c_str() : ""; }

extern "C" const char* hicu_status_string(hicu_status s) {
  switch (s) {
    case HICU_OK: return "HICU_OK";
    case HICU_ERR_ARG: return "HICU_ERR_ARG";
    case HICU_ERR_SHAPE: return "HICU_ERR_SHAPE";
    case HICU_ERR_RANK: return "HICU_ERR_RANK";
    case HICU_ERR_ALLOC: return "HICU_ERR_ALLOC";
    case HICU_ERR_CUDA: return "HICU_ERR_CUDA";
    case HICU_ERR_TIMEOUT: return "HICU_ERR_TIMEOUT";
    case HICU_ERR_NUMERIC: return "HICU_ERR_NUMERIC";
    case HICU_ERR_UNSUPPORTED: return "HICU_ERR_UNSUPPORTED";
  }
  return "HICU_ERR_UNKNOWN";
}

extern "C" hicu_status hicu_check(hicu_handle* h, void* stream) {
  if (!h) return HICU_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(h, e, "stream");
  int err = 0;
  e = cudaMemcpy(&err, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(h, e, "error word");
  if (err) {
    cudaMemset(h->dev_err, 0, sizeof(int));
    return set_error(h, (hicu_status)err, "device-side error recorded");
  }
  return HICU_OK;
}

extern "C" hicu_status hicu_profile_select(hicu_handle* h, int32_t kernel_class) {
  if (!h) return HICU_ERR_ARG;
  if (kernel_class < -1 || kernel_class > K_TRIDIAG)
    return set_error(h, HICU_ERR_ARG, "profile_select: unknown kernel class");
  h->prof_class = kernel_class;
  h->prof_used = 0;
  h->launches_class = 0;
  h->launches_all = 0;
  return HICU_OK;
}

extern "C" hicu_status hicu_profile_read(hicu_handle* h, double* total_ms, int64_t* class_launches,
                                         int64_t* all_launches) {
  if (!h) return HICU_ERR_ARG;
  double ms = 0.0;
  if (h->prof_used > 0) {
    cudaError_t e = cudaEventSynchronize(h->prof_events[h->prof_used - 1]);
    if (e != cudaSuccess) return cuda_error(h, e, "profile_read");
    for (size_t i = 0; i + 1 < h->prof_used; i += 2) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, h->prof_events[i], h->prof_events[i + 1]) == cudaSuccess) ms += t;
    }
  }
  if (total_ms) *total_ms = ms;
  if (class_launches) *class_launches = h->launches_class;
  if (all_launches) *all_launches = h->launches_all;
  h->prof_used = 0;
  h->launches_class = 0;
  h->launches_all = 0;
  return HICU_OK;
}

extern "C" hicu_status hicu_profile_eig_sweeps(hicu_handle* h, int64_t* sweeps) {
  if (!h || !sweeps) return HICU_ERR_ARG;
  unsigned long long v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, h->dev_err + 8, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(h->dev_err + 8, 0, sizeof(v));
  if (e != cudaSuccess) return cuda_error(h, e, "profile_eig_sweeps");
  *sweeps = (int64_t)v;
  return HICU_OK;
}

extern "C" int64_t hicu_filter_length(const hicu_geom* geom) {
  if (!geom_ok(geom)) return -1;
  return (int64_t)geom->ncoil * geom->k[0] * geom->k[1] * geom->k[2];
}

extern "C" int64_t hicu_num_outputs(const hicu_geom* geom, const hicu_region* region) {
  ConvGeom g;
  if (make_conv_geom(nullptr, geom, region, &g) != HICU_OK) return -1;
  return g.s;
}

// ------------------------------------------------------------ hot path

extern "C" hicu_status hicu_gram(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                 const float* x, double* G, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!x || !G) return set_error(h, HICU_ERR_ARG, "gram: null pointer");
  return run_gram(h, geom, region, x, G, (cudaStream_t)stream);
}

extern "C" hicu_status hicu_nullspace(hicu_handle* h, int64_t n, int64_t r, const double* G,
                                      double* Q, double* eigvals, int32_t flags, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!G || !Q) return set_error(h, HICU_ERR_ARG, "nullspace: null pointer");
  if (flags & ~(HICU_NULLSPACE_WARM | HICU_NULLSPACE_SPLIT | HICU_NULLSPACE_GRID | HICU_NULLSPACE_CLUSTER))
    return set_error(h, HICU_ERR_ARG, "nullspace: unknown flags");
  return run_nullspace(h, n, r, G, Q, eigvals, flags, (cudaStream_t)stream);
}

extern "C" hicu_status hicu_principal_subspace(hicu_handle* h, int64_t n, int64_t r, const double* G, double* V,
                                               double* eig_top, double* eig_all, double* tail, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (n < 2 || n > 4096) return set_error(h, HICU_ERR_SHAPE, "principal_subspace: n must be in [2, 4096]");
  if (r <= 0 || r >= n) return set_error(h, HICU_ERR_RANK, "principal_subspace: rank must satisfy 0 < r < n");
  if (!G || !V || !eig_top) return set_error(h, HICU_ERR_ARG, "principal_subspace: null pointer");
  return run_principal(h, n, r, G, V, eig_top, eig_all, tail, (cudaStream_t)stream);
}

extern "C" hicu_status hicu_nullspace_info(hicu_handle* h, int32_t* sweeps, int32_t* converged) {
  if (!h || !sweeps || !converged) return HICU_ERR_ARG;
  if (!h->eig_info) return set_error(h, HICU_ERR_ARG, "nullspace_info: no eigen-decomposition yet");
  int info[4] = {0, 0, 0, 0};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(info, h->eig_info, sizeof(info), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(h, e, "nullspace_info");
  *sweeps = info[0];
  *converged = info[1] ? (info[3] == 1 ? 2 : 1) : 0;
  return HICU_OK;
}

extern "C" hicu_status hicu_jl_compress(hicu_handle* h, int64_t n, int64_t nr, int32_t p,
                                        const double* Q, int32_t mode, const double* P,
                                        uint64_t seed, uint64_t counter, float* filters,
                                        void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!Q || !filters) return set_error(h, HICU_ERR_ARG, "jl_compress: null pointer");
  if (mode != HICU_JL_NULLSPACE && mode != HICU_JL_PROJECTOR && mode != HICU_JL_COMPLEMENT)
    return set_error(h, HICU_ERR_ARG, "jl_compress: unknown mode");
  if (n < 2 || nr < 1 || nr >= n) return set_error(h, HICU_ERR_RANK, "jl_compress: need 1 <= n-r < n");
  if (p < 1 || p > 4096) return set_error(h, HICU_ERR_RANK, "jl_compress: p out of range");
  return launch_jl(h, n, nr, p, Q, mode, P, seed, counter, filters, (cudaStream_t)stream);
}

namespace {

struct StepBuffers {
  float2* fT;
  float2* fA;
  int Ppad, Cpad;
};

hicu_status prep_filters(hicu_handle* h, const ConvGeom& g, const float* bank, int p, bool conv,
                         bool adj, StepBuffers* b, cudaStream_t st) {
  hicu_status s = HICU_OK;
  b->Ppad = conv_ppad(p);
  b->Cpad = adj_cpad(g.C);
  b->fT = conv ? (float2*)ws_get(h, WS_FT, sizeof(float2) * (size_t)g.n * b->Ppad, &s) : nullptr;
  if (s) return s;
  b->fA = adj ? (float2*)ws_get(h, WS_FA, sizeof(float2) * (size_t)g.K * b->Ppad * b->Cpad, &s) : nullptr;
  if (s) return s;
  return launch_prep_filters(h, g, (const float2*)bank, p, b->fT, b->Ppad, b->fA, b->Cpad, st);
}

hicu_status check_prec(hicu_handle* h, int32_t prec) {
  if (prec == HICU_FP32 || prec == HICU_SPLIT_BF16) return HICU_OK;
  return set_error(h, HICU_ERR_ARG, "unknown precision");
}

hicu_status check_tc(hicu_handle* h, const ConvGeom& g) {
  if (tc_supported(g)) return HICU_OK;
  return set_error(h, HICU_ERR_UNSUPPORTED,
                   "split-bf16 path: a circular axis other than the outermost one, or a kernel the "
                   "tensor-core tiling does not fit");
}

}  // namespace

extern "C" hicu_status hicu_conv_null(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                      const float* x, const float* filters, int32_t p, float* R,
                                      double* objective, int32_t prec, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!x || !filters || (!R && !objective)) return set_error(h, HICU_ERR_ARG, "conv_null: null pointer");
  if (p < 1 || p > 4096) return set_error(h, HICU_ERR_RANK, "conv_null: p out of range");
  hicu_status s = check_prec(h, prec);
  if (s) return s;
  ConvGeom g;
  s = make_conv_geom(h, geom, region, &g);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == HICU_SPLIT_BF16) {
    s = check_tc(h, g);
    if (s) return s;
    uint4* xpl = (uint4*)ws_get(h, WS_TC_X, tc_x_bytes(g), &s);
    if (s) return s;
    void* bw = ws_get(h, WS_TC_BC, tc_b_bytes(g, p, 0), &s);
    if (s) return s;
    int nb = 0;
    s = launch_conv_tc(h, g, nullptr, nullptr, p, nullptr, nullptr, nullptr, &nb, st);
    if (s) return s;
    double* part = (double*)ws_get(h, WS_PART, sizeof(double) * nb, &s);
    if (s) return s;
    s = tc_prepare_weights(h, g, (const float2*)filters, p, bw, nullptr, st);
    if (s) return s;
    s = tc_prepare_input(h, g, full_view(geom, region, const_cast<float*>(x)), xpl, st);
    if (s) return s;
    s = launch_conv_tc(h, g, xpl, bw, p, (float2*)R, nullptr, part, &nb, st);
    if (s) return s;
    if (objective) return launch_sum_partials(h, part, nb, objective, st);
    return HICU_OK;
  }
  StepBuffers b;
  s = prep_filters(h, g, filters, p, true, false, &b, st);
  if (s) return s;
  int nb = 0;
  launch_conv_fp32(h, g, full_view(geom, region, const_cast<float*>(x)), b.fT, p, b.Ppad, nullptr,
                   nullptr, &nb, st);
  double* part = (double*)ws_get(h, WS_PART, sizeof(double) * nb, &s);
  if (s) return s;
  s = launch_conv_fp32(h, g, full_view(geom, region, const_cast<float*>(x)), b.fT, p, b.Ppad,
                       (float2*)R, part, &nb, st);
  if (s) return s;
  if (objective) return launch_sum_partials(h, part, nb, objective, st);
  return HICU_OK;
}

extern "C" hicu_status hicu_conv_null_adjoint(hicu_handle* h, const hicu_geom* geom,
                                              const hicu_region* region, const float* R,
                                              const float* filters, int32_t p, const uint8_t* mask,
                                              float* gout, double* gnorm2, int32_t prec,
                                              void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!R || !filters || !gout) return set_error(h, HICU_ERR_ARG, "conv_null_adjoint: null pointer");
  if (p < 1 || p > 4096) return set_error(h, HICU_ERR_RANK, "conv_null_adjoint: p out of range");
  hicu_status s = check_prec(h, prec);
  if (s) return s;
  ConvGeom g;
  s = make_conv_geom(h, geom, region, &g);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  KView gv = full_view(geom, region, gout);
  MView mv = mask_view(geom, region, mask);
  if (prec == HICU_SPLIT_BF16) {
    s = check_tc(h, g);
    if (s) return s;
    uint4* rpl = (uint4*)ws_get(h, WS_TC_R, tc_r_bytes(g, p), &s);
    if (s) return s;
    void* bw = ws_get(h, WS_TC_BA, tc_b_bytes(g, p, 1), &s);
    if (s) return s;
    int nb = 0;
    s = launch_adjoint_tc(h, g, nullptr, nullptr, p, mv, gv, nullptr, &nb, st);
    if (s) return s;
    double* part = (double*)ws_get(h, WS_PART, sizeof(double) * nb, &s);
    if (s) return s;
    s = tc_prepare_weights(h, g, (const float2*)filters, p, nullptr, bw, st);
    if (s) return s;
    s = tc_prepare_r(h, g, (const float2*)R, p, rpl, st);
    if (s) return s;
    s = launch_adjoint_tc(h, g, rpl, bw, p, mv, gv, part, &nb, st);
    if (s) return s;
    if (gnorm2) return launch_sum_partials(h, part, nb, gnorm2, st);
    return HICU_OK;
  }
  StepBuffers b;
  s = prep_filters(h, g, filters, p, false, true, &b, st);
  if (s) return s;
  int nb = 0;
  launch_adjoint_fp32(h, g, (const float2*)R, b.fA, p, b.Ppad, b.Cpad, mv, gv, nullptr, &nb, st);
  double* part = (double*)ws_get(h, WS_PART, sizeof(double) * nb, &s);
  if (s) return s;
  s = launch_adjoint_fp32(h, g, (const float2*)R, b.fA, p, b.Ppad, b.Cpad, mv, gv, part, &nb, st);
  if (s) return s;
  if (gnorm2) return launch_sum_partials(h, part, nb, gnorm2, st);
  return HICU_OK;
}

namespace hicu {

// Split-bf16 tensor-core descent step: conv of y (R kept only as split bf16 planes), masked adjoint,
// conv of g reduced to D, then the same line search and update as the FP32 form.
static hicu_status gd_step_filters_tc(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                      const ConvGeom& g, float* y, const uint8_t* mask, const float* filters,
                                      int p, double* stats, cudaStream_t st, bool planes_valid, bool keep_planes) {
  hicu_status s = check_tc(h, g);
  if (s) return s;
  const size_t xbytes = tc_x_bytes(g);
  uint4* xpl = (uint4*)ws_get(h, WS_TC_X, xbytes, &s);
  if (s) return s;
  uint4* gpl = (uint4*)ws_get(h, WS_TC_G, xbytes, &s);
  if (s) return s;
  uint4* rpl = (uint4*)ws_get(h, WS_TC_R, tc_r_bytes(g, p), &s);
  if (s) return s;
  void* bwc = ws_get(h, WS_TC_BC, tc_b_bytes(g, p, 0), &s);
  if (s) return s;
  void* bwa = ws_get(h, WS_TC_BA, tc_b_bytes(g, p, 1), &s);
  if (s) return s;
  float2* gb = (float2*)ws_get(h, WS_G, sizeof(float2) * (size_t)g.C * g.ex * g.ey * g.ez, &s);
  if (s) return s;
  double* st4 = stats;
  if (!st4) {
    st4 = (double*)ws_get(h, WS_STATS, sizeof(double) * 8, &s);
    if (s) return s;
  }
  const KView yv = full_view(geom, region, y);
  const KView gview = region_view(g, gb);
  const MView mv = mask_view(geom, region, mask);
  int n1 = 0, n2 = 0, n3 = 0;
  s = launch_conv_tc(h, g, nullptr, nullptr, p, nullptr, nullptr, nullptr, &n1, st);
  if (s) return s;
  s = launch_adjoint_tc(h, g, nullptr, nullptr, p, mv, gview, nullptr, &n2, st);
  if (s) return s;
  n3 = n1;
  double* part = (double*)ws_get(h, WS_PART, sizeof(double) * (n1 + n2 + n3), &s);
  if (s) return s;
  if ((s = tc_prepare_weights(h, g, (const float2*)filters, p, bwc, bwa, st))) return s;
  // the split planes of y: left by the previous step's update when the caller says so
  if (!planes_valid && (s = tc_prepare_input(h, g, yv, xpl, st))) return s;
  if ((s = launch_conv_tc(h, g, xpl, bwc, p, nullptr, rpl, part, &n1, st))) return s;
  // the adjoint writes g both as complex64 (for the update) and as the split planes of the
  // line-search convolution's input
  if ((s = launch_adjoint_tc(h, g, rpl, bwa, p, mv, gview, part + n1, &n2, st, gpl))) return s;
  if ((s = launch_conv_tc(h, g, gpl, bwc, p, nullptr, nullptr, part + n1 + n2, &n3, st))) return s;
  if (keep_planes) return launch_update_step_planes(h, g, yv, gview, mv, part, n1, n2, n3, st4, xpl, st);
  if ((s = launch_update_step(h, g, yv, gview, mv, part, n1, n2, n3, st4, st)))
    return cuda_error(h, cudaGetLastError(), "update");
  return HICU_OK;
}

// One descent step for a fixed bank (Algorithm 1 steps 7-8).
hicu_status gd_step_filters(hicu_handle* h, const hicu_geom* geom, const hicu_region* region, float* y,
                            const uint8_t* mask, const float* filters, int32_t p, double* stats,
                            int32_t prec, cudaStream_t st, bool planes_valid,
                            bool keep_planes) {
  hicu_status s = check_prec(h, prec);
  if (s) return s;
  ConvGeom g;
  s = make_conv_geom(h, geom, region, &g);
  if (s) return s;
  if (prec == HICU_SPLIT_BF16)
    return gd_step_filters_tc(h, geom, region, g, y, mask, filters, p, stats, st, planes_valid, keep_planes);
  StepBuffers b;
  s = prep_filters(h, g, filters, p, true, true, &b, st);
  if (s) return s;
  float2* R = (float2*)ws_get(h, WS_R, sizeof(float2) * (size_t)g.s * p, &s);
  if (s) return s;
  float2* gb = (float2*)ws_get(h, WS_G, sizeof(float2) * (size_t)g.C * g.ex * g.ey * g.ez, &s);
  if (s) return s;
  double* st4 = stats;
  if (!st4) {
    st4 = (double*)ws_get(h, WS_STATS, sizeof(double) * 8, &s);
    if (s) return s;
  }
  const KView yv = full_view(geom, region, y);
  const KView gview = region_view(g, gb);
  const MView mv = mask_view(geom, region, mask);
  int n1 = 0, n2 = 0, n3 = 0;
  launch_conv_fp32(h, g, yv, b.fT, p, b.Ppad, nullptr, nullptr, &n1, st);
  launch_adjoint_fp32(h, g, R, b.fA, p, b.Ppad, b.Cpad, mv, gview, nullptr, &n2, st);
  n3 = n1;
  double* part = (double*)ws_get(h, WS_PART, sizeof(double) * (n1 + n2 + n3), &s);
  if (s) return s;
  s = launch_conv_fp32(h, g, yv, b.fT, p, b.Ppad, R, part, &n1, st);
  if (s) return s;
  s = launch_adjoint_fp32(h, g, R, b.fA, p, b.Ppad, b.Cpad, mv, gview, part + n1, &n2, st);
  if (s) return s;
  s = launch_conv_fp32(h, g, gview, b.fT, p, b.Ppad, nullptr, part + n1 + n2, &n3, st);
  if (s) return s;
  s = launch_update_step(h, g, yv, gview, mv, part, n1, n2, n3, st4, st);
  if (s) return cuda_error(h, cudaGetLastError(), "update");
  return HICU_OK;
}

// One descent step with soft data consistency (softdc.cu describes the cost and the step): the
// convolution of y, the unmasked adjoint, the data term added to g on the region, the convolution of
// g, then the update over the whole region.  Partial-sum layout for the update kernel:
// [conv: ||H(y)Q~||^2 | lambda ||M(y - X0)||^2 | ||g||^2 | conv: ||H(g)Q~||^2 | lambda ||M g||^2],
// so its objective, numerator and denominator sums take the data term along.
hicu_status gd_step_filters_soft(hicu_handle* h, const hicu_geom* geom, const hicu_region* region, float* y,
                                 const uint8_t* mask, const float* x0, double lam, const float* filters, int32_t p,
                                 double* stats, int32_t prec, cudaStream_t st) {
  hicu_status s = check_prec(h, prec);
  if (s) return s;
  ConvGeom g;
  s = make_conv_geom(h, geom, region, &g);
  if (s) return s;
  const bool tc = prec == HICU_SPLIT_BF16;
  if (tc && (s = check_tc(h, g))) return s;
  float2* gb = (float2*)ws_get(h, WS_G, sizeof(float2) * (size_t)g.C * g.ex * g.ey * g.ez, &s);
  if (s) return s;
  double* st4 = stats;
  if (!st4) {
    st4 = (double*)ws_get(h, WS_STATS, sizeof(double) * 8, &s);
    if (s) return s;
  }
  const KView yv = full_view(geom, region, y);
  const KView xv = full_view(geom, region, const_cast<float*>(x0));
  const KView gview = region_view(g, gb);
  const MView mv = mask_view(geom, region, mask);
  MView none = mv;
  none.p = nullptr;
  int n1 = 0, n2 = 0, n3 = 0, nb = 0;
  launch_soft_dc(h, g, gview, yv, xv, mv, lam, nullptr, nullptr, nullptr, &nb, st);
  if (tc) {
    const size_t xbytes = tc_x_bytes(g);
    uint4* xpl = (uint4*)ws_get(h, WS_TC_X, xbytes, &s);
    if (s) return s;
    uint4* gpl = (uint4*)ws_get(h, WS_TC_G, xbytes, &s);
    if (s) return s;
    uint4* rpl = (uint4*)ws_get(h, WS_TC_R, tc_r_bytes(g, p), &s);
    if (s) return s;
    void* bwc = ws_get(h, WS_TC_BC, tc_b_bytes(g, p, 0), &s);
    if (s) return s;
    void* bwa = ws_get(h, WS_TC_BA, tc_b_bytes(g, p, 1), &s);
    if (s) return s;
    if ((s = launch_conv_tc(h, g, nullptr, nullptr, p, nullptr, nullptr, nullptr, &n1, st))) return s;
    if ((s = launch_adjoint_tc(h, g, nullptr, nullptr, p, none, gview, nullptr, &n2, st))) return s;
    n3 = n1;
    double* part = (double*)ws_get(h, WS_PART, sizeof(double) * (n1 + n3 + 3 * (size_t)nb + n2), &s);
    if (s) return s;
    double* p_dc = part + n1;
    double* p_g = p_dc + nb;
    double* p_d = p_g + nb;
    double* p_mg = p_d + n3;
    double* p_adj = p_mg + nb;   // the adjoint's own norm partials (not used)
    if ((s = tc_prepare_weights(h, g, (const float2*)filters, p, bwc, bwa, st))) return s;
    if ((s = tc_prepare_input(h, g, yv, xpl, st))) return s;
    if ((s = launch_conv_tc(h, g, xpl, bwc, p, nullptr, rpl, part, &n1, st))) return s;
    if ((s = launch_adjoint_tc(h, g, rpl, bwa, p, none, gview, p_adj, &n2, st))) return s;
    if ((s = launch_soft_dc(h, g, gview, yv, xv, mv, lam, p_dc, p_g, p_mg, &nb, st))) return s;
    if ((s = tc_prepare_input(h, g, gview, gpl, st))) return s;
    if ((s = launch_conv_tc(h, g, gpl, bwc, p, nullptr, nullptr, p_d, &n3, st))) return s;
    if ((s = launch_update_step(h, g, yv, gview, none, part, n1 + nb, nb, n3 + nb, st4, st)))
      return cuda_error(h, cudaGetLastError(), "update");
    return HICU_OK;
  }
  StepBuffers b;
  s = prep_filters(h, g, filters, p, true, true, &b, st);
  if (s) return s;
  float2* R = (float2*)ws_get(h, WS_R, sizeof(float2) * (size_t)g.s * p, &s);
  if (s) return s;
  launch_conv_fp32(h, g, yv, b.fT, p, b.Ppad, nullptr, nullptr, &n1, st);
  launch_adjoint_fp32(h, g, R, b.fA, p, b.Ppad, b.Cpad, none, gview, nullptr, &n2, st);
  n3 = n1;
  double* part = (double*)ws_get(h, WS_PART, sizeof(double) * (n1 + n3 + 3 * (size_t)nb + n2), &s);
  if (s) return s;
  double* p_dc = part + n1;
  double* p_g = p_dc + nb;
  double* p_d = p_g + nb;
  double* p_mg = p_d + n3;
  double* p_adj = p_mg + nb;
  if ((s = launch_conv_fp32(h, g, yv, b.fT, p, b.Ppad, R, part, &n1, st))) return s;
  if ((s = launch_adjoint_fp32(h, g, R, b.fA, p, b.Ppad, b.Cpad, none, gview, p_adj, &n2, st))) return s;
  if ((s = launch_soft_dc(h, g, gview, yv, xv, mv, lam, p_dc, p_g, p_mg, &nb, st))) return s;
  if ((s = launch_conv_fp32(h, g, gview, b.fT, p, b.Ppad, nullptr, p_d, &n3, st))) return s;
  if ((s = launch_update_step(h, g, yv, gview, none, part, n1 + nb, nb, n3 + nb, st4, st)))
    return cuda_error(h, cudaGetLastError(), "update");
  return HICU_OK;
}

}  // namespace hicu

extern "C" hicu_status hicu_gd_step_soft(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                         float* y, const uint8_t* mask, const float* x0, double lambda,
                                         const float* filters, int32_t p, double* stats, int32_t prec, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!y || !mask || !x0 || !filters) return set_error(h, HICU_ERR_ARG, "gd_step_soft: null pointer");
  if (p < 1 || p > 4096) return set_error(h, HICU_ERR_RANK, "gd_step_soft: p out of range");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return set_error(h, HICU_ERR_ARG, "gd_step_soft: lambda must be >= 0");
  return gd_step_filters_soft(h, geom, region, y, mask, x0, lambda, filters, p, stats, prec, (cudaStream_t)stream);
}

extern "C" hicu_status hicu_gd_step_filters(hicu_handle* h, const hicu_geom* geom,
                                            const hicu_region* region, float* y, const uint8_t* mask,
                                            const float* filters, int32_t p, double* stats,
                                            int32_t prec, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!y || !filters) return set_error(h, HICU_ERR_ARG, "gd_step_filters: null pointer");
  if (p < 1 || p > 4096) return set_error(h, HICU_ERR_RANK, "gd_step_filters: p out of range");
  return gd_step_filters(h, geom, region, y, mask, filters, p, stats, prec, (cudaStream_t)stream);
}

extern "C" hicu_status hicu_gd_step(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                    float* y, const uint8_t* mask, const double* Q, int64_t nr,
                                    int32_t p, int32_t jl_mode, uint64_t seed, uint64_t counter,
                                    const double* P, double* stats, int32_t prec, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!y || !Q) return set_error(h, HICU_ERR_ARG, "gd_step: null pointer");
  const int64_t n = hicu_filter_length(geom);
  if (n < 0) return set_error(h, HICU_ERR_SHAPE, "gd_step: invalid geometry");
  if (nr < 1 || nr >= n) return set_error(h, HICU_ERR_RANK, "gd_step: need 1 <= n-r < n");
  if (p < 1 || p > 4096) return set_error(h, HICU_ERR_RANK, "gd_step: p out of range");
  if (jl_mode == HICU_JL_NULLSPACE && p > nr)
    return set_error(h, HICU_ERR_RANK, "gd_step: p must not exceed n-r");
  hicu_status s = HICU_OK;
  float* bank = (float*)ws_get(h, WS_BANK, sizeof(float2) * (size_t)p * n, &s);
  if (s) return s;
  s = hicu_jl_compress(h, n, nr, p, Q, jl_mode, P, seed, counter, bank, stream);
  if (s) return s;
  return gd_step_filters(h, geom, region, y, mask, bank, p, stats, prec, (cudaStream_t)stream);
}

// ------------------------------------------------------------- reconstruct

namespace {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// time-averaged start along z (2D+t): unsampled (c, y, x, t) take the mean of the
// sampled frames at (c, y, x), or zero if none was sampled
__global__ void time_average_kernel(int C, int nx, int ny, int nz, float2* x, const uint8_t* m,
                                    long long msc) {
  const long long tot = (long long)C * ny * nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nx);
    const int iy = (int)((i / nx) % ny);
    const int c = (int)(i / ((long long)nx * ny));
    const long long plane = (long long)nx * ny;
    double sr = 0.0, si = 0.0;
    int cnt = 0;
    for (int z = 0; z < nz; ++z) {
      const long long o = z * plane + (long long)iy * nx + ix;
      if (m[c * msc + o]) {
        const float2 v = x[c * plane * nz + o];
        sr += v.x;
        si += v.y;
        ++cnt;
      }
    }
    const float2 avg = cnt ? make_float2((float)(sr / cnt), (float)(si / cnt)) : make_float2(0.f, 0.f);
    for (int z = 0; z < nz; ++z) {
      const long long o = z * plane + (long long)iy * nx + ix;
      if (!m[c * msc + o]) x[c * plane * nz + o] = avg;
    }
  }
}

__global__ void tail_sum_kernel(const double* eig, int nr, double* out) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < nr; i += 256) s += eig[i];
  s = block_sum<256>(s, sh);
  if (threadIdx.x == 0) *out = s;
}

}  // namespace

// A host input goes up in two parts: the z planes of the first stage's region (every channel) on
// the call's stream, then the other planes on the handle's copy stream while the first stages run,
// which read and write y only inside their regions.  The call's stream waits for the second part
// before the first stage that reaches beyond those planes and before the output copy, and on an
// early return, so that synchronising the call's stream always covers the copy.
struct StagedUpload {
  hicu_handle* h;
  cudaStream_t st;
  long long z0, z1;   // planes uploaded on the call's stream
  bool pending = false;
  bool covers(const hicu_region& r) const { return r.off[2] >= z0 && r.off[2] + r.ext[2] <= z1; }
  hicu_status join() {
    if (!pending) return HICU_OK;
    pending = false;
    return cuda_error(h, cudaStreamWaitEvent(st, h->copy_join, 0), "reconstruct: upload join");
  }
  ~StagedUpload() {
    if (pending) cudaStreamWaitEvent(st, h->copy_join, 0);
  }
};

extern "C" hicu_status hicu_reconstruct(hicu_handle* h, const hicu_geom* geom, const float* x0,
                                        const uint8_t* mask, const hicu_params* prm, float* x_out,
                                        hicu_log* log, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!geom || !x0 || !mask || !prm || !x_out) return set_error(h, HICU_ERR_ARG, "reconstruct: null pointer");
  if (!geom_ok(geom)) return set_error(h, HICU_ERR_SHAPE, "reconstruct: invalid geometry");
  if (prm->nstages < 1 || !prm->stages) return set_error(h, HICU_ERR_ARG, "reconstruct: no stages");
  cudaStream_t st = (cudaStream_t)stream;
  // kernel mask: the null space lives on the C |K| coefficients of the support, the convolutions
  // on the box (n_box) with the bank scattered into it
  const int64_t n_box = hicu_filter_length(geom);
  const int* sup = nullptr;
  const int* inv = nullptr;
  int nk = 0;
  if (prm->kernel_mask) {
    hicu_status sm = support_maps(h, geom, prm->kernel_mask, &sup, &inv, &nk, st);
    if (sm) return sm;
  }
  const int64_t n = prm->kernel_mask ? (int64_t)geom->ncoil * nk : n_box;
  const int64_t r = prm->rank;
  if (r < 1 || r >= n) return set_error(h, HICU_ERR_RANK, "reconstruct: rank must satisfy 0 < r < n");
  const int64_t nr = n - r;
  if (prm->jl != HICU_JL_NULLSPACE && prm->jl != HICU_JL_PROJECTOR)
    return set_error(h, HICU_ERR_ARG, "reconstruct: unknown JL mode");
  if (prm->init != 0 && prm->init != 1) return set_error(h, HICU_ERR_ARG, "reconstruct: unknown init");
  if (!(prm->dc_weight >= 0.0) || !std::isfinite(prm->dc_weight) || !(prm->l1_threshold >= 0.0) ||
      !std::isfinite(prm->l1_threshold))
    return set_error(h, HICU_ERR_ARG, "reconstruct: dc_weight and l1_threshold must be finite and >= 0");
  if (prm->eig_solver != 0 && prm->eig_solver != HICU_NULLSPACE_GRID && prm->eig_solver != HICU_NULLSPACE_CLUSTER &&
      prm->eig_solver != HICU_NULLSPACE_TRIDIAG && prm->eig_solver != HICU_NULLSPACE_RSVD)
    return set_error(h, HICU_ERR_ARG, "reconstruct: unknown eig_solver");
  if ((prm->eig_solver == HICU_NULLSPACE_TRIDIAG || prm->eig_solver == HICU_NULLSPACE_RSVD) &&
      prm->jl != HICU_JL_PROJECTOR)
    return set_error(h, HICU_ERR_ARG, "reconstruct: the principal-vector solvers need jl = HICU_JL_PROJECTOR");
  // principal vectors V and complement filters (I - V V^H) P: the projector-mode filters
  const bool principal = prm->jl == HICU_JL_PROJECTOR && (prm->eig_solver == 0 || prm->eig_solver == HICU_NULLSPACE_TRIDIAG ||
                                                          prm->eig_solver == HICU_NULLSPACE_RSVD);
  const bool rsvd = prm->eig_solver == HICU_NULLSPACE_RSVD;
  hicu_status s = check_prec(h, prm->prec);
  if (s) return s;
  long long total_iters = 0, total_steps = 0;
  for (int i = 0; i < prm->nstages; ++i) {
    const hicu_stage& stg = prm->stages[i];
    ConvGeom g;
    s = make_conv_geom(h, geom, &stg.region, &g);
    if (s) return s;
    if (stg.iters < 0 || stg.gd_steps < 0) return set_error(h, HICU_ERR_ARG, "reconstruct: negative count");
    if (!prm->jl_exact && (stg.p < 1 || (prm->jl == HICU_JL_NULLSPACE && stg.p > nr)))
      return set_error(h, HICU_ERR_RANK, "reconstruct: p must be in [1, n-r]");
    total_iters += stg.iters;
    total_steps += (long long)stg.iters * stg.gd_steps;
  }
  const long long N = geom->dim[0] * geom->dim[1] * geom->dim[2] * (long long)geom->ncoil;
  const long long NM = geom->dim[0] * geom->dim[1] * geom->dim[2] * (geom->mask_per_coil ? geom->ncoil : 1);
  const bool out_dev = is_device_ptr(x_out);
  const bool in_dev = is_device_ptr(x0);
  const bool m_dev = is_device_ptr(mask);
  float* y = x_out;
  if (!out_dev) {
    y = (float*)ws_get(h, WS_REC_X, sizeof(float2) * N, &s);
    if (s) return s;
  }
  const uint8_t* m = mask;
  if (!m_dev) {
    uint8_t* mm = (uint8_t*)ws_get(h, WS_REC_M, NM, &s);
    if (s) return s;
    if (cudaMemcpyAsync(mm, mask, NM, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return cuda_error(h, cudaGetLastError(), "reconstruct: mask upload");
    m = mm;
  }
  const bool soft = prm->dc_weight > 0.0, l1 = prm->l1_threshold > 0.0;
  // a host input is uploaded in two parts where the first stage covers only some z planes and
  // nothing reads the whole array first (time-averaged start, a copy of X0); a circular z axis
  // goes up whole
  const long long Z = geom->dim[2];
  StagedUpload up{h, st, 0, Z};
  if (!in_dev && !geom->circular[2] && prm->init == 0 && !soft && !l1) {
    up.z0 = prm->stages[0].region.off[2];
    up.z1 = up.z0 + prm->stages[0].region.ext[2];
  }
  if (up.z0 == 0 && up.z1 == Z) {
    if (cudaMemcpyAsync(y, x0, sizeof(float2) * N, in_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return cuda_error(h, cudaGetLastError(), "reconstruct: input copy");
  } else {
    if ((s = ensure_copy_stream(h))) return s;
    const size_t pbytes = sizeof(float2) * (size_t)(geom->dim[0] * geom->dim[1]);   // one z plane
    char* yd = reinterpret_cast<char*>(y);
    const char* xs = reinterpret_cast<const char*>(x0);
    auto part = [&](long long c, long long za, long long zb, cudaStream_t cs) {
      const size_t off = (size_t)(c * Z + za) * pbytes;
      return za < zb ? cudaMemcpyAsync(yd + off, xs + off, (size_t)(zb - za) * pbytes, cudaMemcpyHostToDevice, cs)
                     : cudaSuccess;
    };
    cudaError_t ce = cudaSuccess;
    for (long long c = 0; c < geom->ncoil && ce == cudaSuccess; ++c) ce = part(c, up.z0, up.z1, st);
    if (ce == cudaSuccess) ce = cudaEventRecord(h->copy_fork, st);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h->copy_st, h->copy_fork, 0);
    if (ce != cudaSuccess) return cuda_error(h, ce, "reconstruct: input copy");
    for (long long c = 0; c < geom->ncoil && ce == cudaSuccess; ++c) {
      ce = part(c, 0, up.z0, h->copy_st);
      if (ce == cudaSuccess) ce = part(c, up.z1, Z, h->copy_st);
    }
    const cudaError_t cj = cudaEventRecord(h->copy_join, h->copy_st);
    if (cj != cudaSuccess) {
      cudaStreamSynchronize(h->copy_st);   // nothing to join: the copies end before the return
      return cuda_error(h, cj, "reconstruct: input copy");
    }
    up.pending = true;
    if (ce != cudaSuccess) return cuda_error(h, ce, "reconstruct: input copy");
  }
  // the observed data X0, kept for the soft data-consistency term and for restoring the samples after
  // the l1 step (the start estimate in y may differ from it: time-averaged initialisation)
  float* x0c = nullptr;
  if (soft || l1) {
    x0c = (float*)ws_get(h, WS_REC_X0, sizeof(float2) * N, &s);
    if (s) return s;
    if (cudaMemcpyAsync(x0c, y, sizeof(float2) * N, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return cuda_error(h, cudaGetLastError(), "reconstruct: X0 copy");
  }
  double* G = (double*)ws_get(h, WS_REC_G, sizeof(double2) * n * n, &s);
  if (s) return s;
  double* Q = (double*)ws_get(h, WS_REC_Q, sizeof(double2) * n * (principal ? r : nr), &s);
  if (s) return s;
  double* eig = (double*)ws_get(h, WS_REC_EIG, sizeof(double) * n, &s);
  if (s) return s;
  double* dlog = (double*)ws_get(h, WS_REC_LOG, sizeof(double) * (total_iters + 1), &s);
  if (s) return s;
  double* dstats = (double*)ws_get(h, WS_REC_STATS, sizeof(double) * 4 * (total_steps + 1), &s);
  if (s) return s;
  if (prm->jl_exact != 0 && prm->jl_exact != 1) return set_error(h, HICU_ERR_ARG, "reconstruct: jl_exact is 0 or 1");
  // augmented null space [Q | Q+], Q+ = blockdiag(Q0, ...) over qplus_blocks groups of channels
  const bool aug = prm->qplus != nullptr;
  int n0 = 0, m0 = 0;
  if (aug) {
    const int nb = prm->qplus_blocks;
    m0 = prm->qplus_cols;
    if (nb < 1 || m0 < 1 || geom->ncoil % nb != 0)
      return set_error(h, HICU_ERR_SHAPE, "reconstruct: qplus_blocks must divide the channels, qplus_cols >= 1");
    n0 = (int)(n / nb);
    if ((int64_t)n0 * nb != n || m0 > n0)
      return set_error(h, HICU_ERR_SHAPE, "reconstruct: Q0 must have n / qplus_blocks rows and at most as many columns");
  }
  const int64_t mplus = aug ? (int64_t)prm->qplus_blocks * m0 : 0;
  // the JL basis (principal vectors, or the null basis), its matrices' row count (with the rows
  // that multiply Q+), and with jl_exact the filter count of the uncompressed gradient (identity
  // P: Q~ = [I - V V^H | Q+], or [Q | Q+])
  const int64_t nq = principal ? r : nr;
  const int jmode = principal ? HICU_JL_COMPLEMENT : prm->jl;
  const int64_t prow0 = (jmode == HICU_JL_NULLSPACE) ? nq : n;
  const int64_t prow = prow0 + mplus;
  const int p_exact = (int)prow;
  float2* q0f = nullptr;
  if (aug) {
    q0f = (float2*)ws_get(h, WS_QPLUS, sizeof(float2) * (size_t)n0 * m0, &s);
    if (s) return s;
    float2* tmp = nullptr;
    if ((s = jl_convert_q(h, n0, m0, prm->qplus, &tmp, st))) return s;
    if (cudaMemcpyAsync(q0f, tmp, sizeof(float2) * (size_t)n0 * m0, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return cuda_error(h, cudaGetLastError(), "reconstruct: Q0 copy");
  }
  int pmax = 1;
  for (int i = 0; i < prm->nstages; ++i) pmax = std::max(pmax, prm->jl_exact ? p_exact : (int)prm->stages[i].p);
  float* bank = (float*)ws_get(h, WS_BANK, sizeof(float2) * (size_t)pmax * n_box, &s);
  if (s) return s;
  float* bank_sup = nullptr;   // JL filters on the support of the kernel mask, before the scatter
  if (prm->kernel_mask) {
    bank_sup = (float*)ws_get(h, WS_BANK_SUP, sizeof(float2) * (size_t)pmax * n, &s);
    if (s) return s;
  }
  if (prm->init == 1) {
    HICU_LAUNCH(h, K_MISC, st,
                time_average_kernel<<<1024, 256, 0, st>>>(
                    geom->ncoil, (int)geom->dim[0], (int)geom->dim[1], (int)geom->dim[2], (float2*)y, m,
                    geom->mask_per_coil ? geom->dim[0] * geom->dim[1] * geom->dim[2] : 0));
  }
  size_t pbatch = 0;
  for (int i = 0; i < prm->nstages; ++i)
    pbatch = std::max(pbatch, (size_t)prm->stages[i].gd_steps * (size_t)prow * (size_t)prm->stages[i].p);
  if (prm->jl_exact) pbatch = (size_t)prow * prow;
  float* Pall = nullptr;
  if (pbatch > 0) {
    Pall = (float*)ws_get(h, WS_REC_P, sizeof(float) * pbatch, &s);
    if (s) return s;
    if ((s = ensure_side_stream(h))) return s;
    if (prm->jl_exact && (s = jl_identity(h, prow, Pall, st))) return s;
  }
  uint64_t counter = 0;
  long long it = 0;
  hicu_region prev = prm->stages[0].region;
  for (int si = 0; si < prm->nstages; ++si) {
    const hicu_stage& stg = prm->stages[si];
    if (!up.covers(stg.region) && (s = up.join())) return s;
    // split planes of y on this stage's region: made by the stage's first step, then kept current
    // by each step's update (the Gram and eigen-solve leave y alone)
    bool planes_valid = false;
    bool whole = true;
    for (int a = 0; a < 3; ++a) whole = whole && stg.region.off[a] == 0 && stg.region.ext[a] == geom->dim[a];
    for (int i = 0; i < stg.iters; ++i) {
      // the JL matrices of this outer iteration's descent steps depend on nothing but the seed and
      // the step counter: drawn on the side stream beside the Gram and the eigen-solve (after the
      // previous iteration's steps, the last readers of the buffer)
      const int pst = prm->jl_exact ? p_exact : stg.p;   // filters per descent step
      if (stg.gd_steps > 0 && !prm->jl_exact) {
        cudaError_t ce = cudaEventRecord(h->draw_fork, st);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h->side_st, h->draw_fork, 0);
        if (ce != cudaSuccess) return cuda_error(h, ce, "reconstruct: draw fork");
        if ((s = jl_draw(h, prow, stg.p, stg.gd_steps, prm->seed, counter, Pall, h->side_st))) return s;
        if ((ce = cudaEventRecord(h->draw_join, h->side_st)) != cudaSuccess)
          return cuda_error(h, ce, "reconstruct: draw join");
      }
      const hicu_region& greg = prm->gram_on_current ? stg.region : prev;
      if (rsvd) {
        // randomized SVD of H on the previous region, warm-started from the last principal vectors
        const int64_t l = prm->rsvd_cols > 0 ? prm->rsvd_cols : std::min<int64_t>(n, r + std::max<int64_t>(r / 2, 8));
        s = run_rsvd(h, geom, &greg, prm->kernel_mask, y, r, l, it > 0 ? Q : nullptr, it > 0 ? r : 0, prm->rsvd_seed,
                     (uint64_t)it, Q, eig, dlog + it, st);
        if (s) return s;
      } else {
        s = run_gram(h, geom, &greg, y, G, st, sup, nk);
        if (s) return s;
      }
      // after the first outer iteration: warm start, and stop at the top-r / rest split (step 3
      // needs an orthonormal basis of the complement of the r principal vectors, nothing more)
      if (rsvd) {
        // V and J came from the randomized SVD
      } else if (principal) {
        // Q (here: the r principal vectors) and J of Eq. 1 directly
        s = run_principal(h, n, r, G, Q, eig, nullptr, dlog + it, st);
        if (s) return s;
      } else {
        s = run_nullspace(h, n, r, G, Q, eig,
                          HICU_NULLSPACE_SPLIT | (it > 0 ? HICU_NULLSPACE_WARM : 0) | prm->eig_solver, st);
        if (s) return s;
        HICU_LAUNCH(h, K_MISC, st, tail_sum_kernel<<<1, 256, 0, st>>>(eig, (int)nr, dlog + it));
      }
      // Algorithm 1 steps 6-8: the basis is converted to complex64 once per outer iteration
      float2* Qf = nullptr;
      if (stg.gd_steps > 0) {
        if ((s = jl_convert_q(h, n, nq, Q, &Qf, st))) return s;
        if (!prm->jl_exact) {
          const cudaError_t ce = cudaStreamWaitEvent(st, h->draw_join, 0);
          if (ce != cudaSuccess) return cuda_error(h, ce, "reconstruct: draw wait");
        }
      }
      for (int j = 0; j < stg.gd_steps; ++j) {
        const float* Pj = prm->jl_exact ? Pall : Pall + (size_t)j * prow * stg.p;
        float* bank_j = prm->kernel_mask ? bank_sup : bank;
        s = launch_jl_converted(h, n, nq, pst, Qf, jmode, nullptr, Pj, prm->seed, counter, bank_j, st, j > 0);
        if (s) return s;
        // rows prow0 .. prow-1 of the step's JL matrix multiply Q+
        if (aug && (s = launch_jl_qplus(h, pst, n, n0, m0, q0f, Pj + (size_t)prow0 * pst, bank_j, st))) return s;
        if (prm->kernel_mask &&
            (s = launch_support_scatter(h, pst, geom->ncoil, geom->k[0] * geom->k[1] * geom->k[2], nk, inv,
                                        (const float2*)bank_sup, (float2*)bank, st)))
          return s;
        if (soft) {
          s = gd_step_filters_soft(h, geom, &stg.region, y, m, x0c, prm->dc_weight, bank, pst,
                                   dstats + 4 * counter, prm->prec, st);
        } else {
          // the update leaves the split planes of y for the next step of the same region
          s = gd_step_filters(h, geom, &stg.region, y, m, bank, pst, dstats + 4 * counter, prm->prec, st,
                              planes_valid, true);
          planes_valid = true;
        }
        if (s) return s;
        // the l1 step after Algorithm 1 step 8, on stages over the whole array; under hard data
        // consistency the observed samples are restored after it
        if (l1 && whole) {
          if ((s = run_soft_threshold(h, geom, y, prm->l1_threshold, st))) return s;
          if (!soft && (s = launch_restore_observed(h, geom, y, x0c, m, st))) return s;
          planes_valid = false;
        }
        ++counter;
      }
      ++it;
      prev = stg.region;
    }
  }
  if ((s = up.join())) return s;
  if (!out_dev) {
    if (cudaMemcpyAsync(x_out, y, sizeof(float2) * N, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return cuda_error(h, cudaGetLastError(), "reconstruct: output copy");
  }
  if (log) {
    std::vector<double> hs(4 * (total_steps + 1));
    if (log->J &&
        cudaMemcpyAsync(log->J, dlog, sizeof(double) * total_iters, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return cuda_error(h, cudaGetLastError(), "reconstruct: log copy");
    if (cudaMemcpyAsync(hs.data(), dstats, sizeof(double) * 4 * total_steps, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
      return cuda_error(h, cudaGetLastError(), "reconstruct: log copy");
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_error(h, cudaGetLastError(), "reconstruct: sync");
    for (long long k = 0; k < total_steps; ++k) {
      if (log->eta) log->eta[k] = hs[4 * k];
      if (log->objective) log->objective[k] = hs[4 * k + 1];
    }
  }
  if (!out_dev || log) return hicu_check(h, stream);
  return cuda_error(h, cudaGetLastError(), "reconstruct");
}
