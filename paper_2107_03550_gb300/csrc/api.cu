// C ABI of libsbiem: handle life cycle, tables, step enqueueing and I/O.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"
#include "mlp.cuh"
#include "sbiem.h"

using namespace sbiem;

namespace sbiem {
int mlp_deploy(const float* params_host, MlpDev* dst, cudaStream_t st);
}

namespace {

thread_local std::string g_last_error;

// Sweep shape of a new handle (chunk length x stages in flight).
constexpr int kDefaultSweepShape = 3;
// Largest on-chip weight table (bytes): it is read through L1 beside the
// sweep's stages in shared memory.
constexpr int64_t kGenMaxTableBytes = 64 * 1024;
// Modes whose s step is at most this evaluate their weights on chip by
// default (the largest step the sweep's blocks of eight lags allow); the
// autotuner revisits it.
constexpr float kGenDsMaxDefault = static_cast<float>(kGenDsBlockMax);

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(SBIEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)


}  // namespace

struct sbiem_s {
  sbiem_params p{};
  int device = 0;
  int sm_count = 0;
  int hist_grid = 0;  // resident CTAs of the history convolution
  cudaStream_t stream = nullptr;      // where work is enqueued
  cudaStream_t own = nullptr;         // the handle's own stream (also used for graph capture)
  bool user_stream = false;
  int N = 0, nmodes = 0;
  double L = 0, dt_min = 0, S = 0, eta = 0;
  std::vector<int64_t> M, Rn, ring_off, w_off;
  std::vector<int64_t> MT, MN;        // the shear and normal kernels' own windows (M = max)
  int64_t total_slots = 0, total_w = 0;
  std::vector<Chunk> chunks;
  std::vector<void*> allocs;
  int64_t device_bytes = 0;
  DevFault<double> f64{};
  DevFault<float> f32{};
  FftGeom g64{};
  double2 *u_a = nullptr, *u_b = nullptr, *u_c = nullptr;  // FP64 utility buffers
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  unsigned* h_status = nullptr;  // pinned
  long long* h_steps = nullptr;  // pinned
  std::map<int, cudaGraphExec_t> graphs;
  std::map<int, cudaGraph_t> graph_defs;
  // overlapped form: the history sweep of the next step runs on a side
  // stream during this step's passes; lag_m is the step length (in dt_min)
  // for which AT/AN already hold the next step's sums (-1: none)
  std::map<int, cudaGraphExec_t> lag_graphs;
  std::map<int, cudaGraph_t> lag_defs;
  // sbiem_step_host with pinned host buffers: the copies in, the overlapped
  // step and the copies out (result, status word) as one graph, captured for
  // one step length and one pair of host pointers
  struct {
    int m = 0;
    const void* tau = nullptr;
    void* V = nullptr;
    cudaGraph_t def = nullptr;
    cudaGraphExec_t exec = nullptr;
  } host_graph;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_started = nullptr;  // every CTA of the step's first pass kernel has started
  int lag_m = -1;
  int lag_grid = 0;  // CTAs of the overlapped sweep (leaves room for the passes)
  int sweep_shape = 0;  // chunk length x stages of the sweep
  int lag_shape = 0;    // the same for the overlapped sweep
  int sweep_ctas = 0;   // resident sweep CTAs per SM asked for (0: as many as fit)
  int lag_ctas = 0;     // the same for the overlapped sweep (0: the rule of sweep_config)
  long long spin_limit = SBIEM_WAIT_LIMIT_DEFAULT;  // polls of the sweep's consumer waits
  // output of sbiem_run: callback, its argument, every how many accepted
  // steps, and page-locked host copies of slip and slip rate
  sbiem_output_fn out_cb = nullptr;
  void* out_user = nullptr;
  int64_t out_every = 0;
  double* h_out = nullptr;  // 2N
  // device footprint planned at creation (for the out-of-memory message)
  int64_t planned_bytes = 0, planned_ring = 0, planned_w = 0;
  int gen_pieces = 0;   // pieces of the on-chip weight table (0: none, weights streamed)
  float gen_ds_max = 0;  // modes with ds = c_s k_n dt_min <= this evaluate their weights on chip
  double gen_err = 0.0; // its largest error relative to dt max|C|
  // timing probe: 4 events per slot; graph event-record nodes are retargeted
  // to the slot of each launch
  int pslots = 0;
  int64_t pcount = 0;
  int pcur = 0;
  std::vector<cudaEvent_t> pev;
  std::map<int, std::vector<cudaGraphNode_t>> pnodes;  // per graph: nodes of marks 0..3
  int64_t chunk_slots = 2048;
  // adaptive run (Sec. 3.2): snapshot of the state, undo copy of ring slots
  double* snap = nullptr;        // V, xV, psi, thd, delta, theta (6N) + t
  double2* snap_spec = nullptr;  // dhat, khat
  int32_t* snap_head = nullptr;
  long long* snap_steps = nullptr;
  void* tune_slots = nullptr;   // one ring slot per mode (the autotuner's timed steps)
  void* undo = nullptr;          // ring-sized
  double* dfull = nullptr;
  double* d_err = nullptr;
  MlpDev* mlp = nullptr;         // deployed Newton initial-guess network
  float* harvest = nullptr;
  unsigned long long* harvest_count = nullptr;
  int64_t harvest_cap = 0;

  bool fp32() const { return p.precision == 1; }
};

namespace {

void* dev_alloc(sbiem_s* s, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* ptr = nullptr;
  if (s->p.alloc_fn) {
    ptr = s->p.alloc_fn(bytes, s->p.alloc_user);
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    ptr = nullptr;
  }
  if (ptr) {
    s->allocs.push_back(ptr);
    s->device_bytes += static_cast<int64_t>(bytes);
    cudaMemsetAsync(ptr, 0, bytes, s->stream);
  }
  return ptr;
}

template <class T>
T* alloc_n(sbiem_s* s, size_t n, bool* ok) {
  T* ptr = static_cast<T*>(dev_alloc(s, n * sizeof(T)));
  if (!ptr) *ok = false;
  return ptr;
}

// SBIEM_ERR_NOMEM with the footprint the handle needs: rings, weights and
// the element and spectral arrays (planned before the first allocation),
// and what was allocated before the failure.
int nomem(const sbiem_s* s, const char* what) {
  char buf[320];
  std::snprintf(buf, sizeof(buf),
                "device allocation failed (%s): the handle needs about %.3f GB (history rings %.3f GB, "
                "weights %.3f GB); %.3f GB were allocated before the failure",
                what, s->planned_bytes / 1e9, s->planned_ring / 1e9, s->planned_w / 1e9, s->device_bytes / 1e9);
  return fail(SBIEM_ERR_NOMEM, buf);
}

void drop_host_graph(sbiem_s* s) {
  if (s->host_graph.exec) cudaGraphExecDestroy(s->host_graph.exec);
  if (s->host_graph.def) cudaGraphDestroy(s->host_graph.def);
  s->host_graph.exec = nullptr;
  s->host_graph.def = nullptr;
  s->host_graph.m = 0;
}

void free_all(sbiem_s* s) {
  drop_host_graph(s);
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : s->graph_defs) cudaGraphDestroy(kv.second);
  for (auto& kv : s->lag_graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : s->lag_defs) cudaGraphDestroy(kv.second);
  s->graphs.clear();
  s->graph_defs.clear();
  s->lag_graphs.clear();
  s->lag_defs.clear();
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->side) cudaStreamSynchronize(s->side);
  for (auto& e : s->pev)
    if (e) cudaEventDestroy(e);
  s->pev.clear();
  for (void* ptr : s->allocs) {
    if (s->p.free_fn) s->p.free_fn(ptr, s->p.alloc_user);
    else cudaFree(ptr);
  }
  s->allocs.clear();
  if (s->h_out) cudaFreeHost(s->h_out);
  if (s->h_status) cudaFreeHost(s->h_status);
  if (s->h_steps) cudaFreeHost(s->h_steps);
  if (s->own) cudaStreamDestroy(s->own);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->ev_started) cudaEventDestroy(s->ev_started);
}

bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

// Windows of the truncated convolution (Sec. 3.1): T_w = eta Omega / cs for
// k <= k_c, (eta Omega / cs)(k_c / k) above; M_n = ceil(T_w / dt_min) with a
// relative slack of 1e-12 against rounding of exact ratios; M_0 = 0.  The
// shear kernel is cut at k_c = kc_L / (eta Omega), the normal kernel at
// kcN_L / (eta Omega) when kcN_L > 0 (the two cutting planes of Sec. 3.1);
// the rings keep M = max(M^T, M^N) lags.  eta = 0 is the quasi-dynamic limit
// (Appendix, Quasi-dynamic BIEM): every window empty, so no history and no
// current-interval kernel term.
void windows_one(const sbiem_params& p, double kc_L, double L, double dt_min, std::vector<int64_t>& M) {
  const int64_t nm = p.N / 2 + 1;
  M.assign(nm, 0);
  if (p.eta_w == 0.0) return;
  double kc = kc_L / (p.eta_w * L);
  if (p.kc_units == 1) kc *= 2.0 * M_PI;
  for (int64_t n = 1; n < nm; ++n) {
    const double k = 2.0 * M_PI * static_cast<double>(n) / L;
    double Tw = p.eta_w * L / p.cs;
    if (k > kc) Tw *= kc / k;
    M[n] = static_cast<int64_t>(std::ceil(Tw / dt_min * (1.0 - 1e-12)));
  }
}

void windows(const sbiem_params& p, double L, double dt_min, std::vector<int64_t>& M, std::vector<int64_t>& MT,
             std::vector<int64_t>& MN) {
  windows_one(p, p.kc_L, L, dt_min, MT);
  if (p.kcN_L > 0.0) windows_one(p, p.kcN_L, L, dt_min, MN);
  else MN = MT;
  M.resize(MT.size());
  for (size_t n = 0; n < MT.size(); ++n) M[n] = std::max(MT[n], MN[n]);
}

// Grids and shapes of the two sweeps from sweep_shape, the weight form and
// the CTAs per SM asked for.  Beside the one-launch FP32 pass the overlapped
// sweep leaves each SM room for the pass kernels: with 2048-lag chunks
// (shapes 3 and 4) shape 4 (one stage) on two CTAs per SM (with two stages
// only one fits beside a pass CTA; flushed N = 4096 steps: 48-50 us with
// one CTA per SM of the on-chip weight form, 41 us with two of the streamed
// form); other shapes
// one CTA per SM; with the four-kernel FFT (small CTAs) the full grid.
void sweep_config(sbiem_s* s) {
  const bool gen = s->fp32() && s->f32.wtab && s->gen_ds_max > 0.0f;
  s->f32.gen_ds_max = gen ? s->gen_ds_max : 0.0f;
  int per_sm = s->fp32() ? sweep_blocks_per_sm<float>(s->sweep_shape, gen)
                         : sweep_blocks_per_sm<double>(s->sweep_shape, false);
  if (per_sm < 1) per_sm = 1;
  if (s->sweep_ctas > 0 && s->sweep_ctas < per_sm) per_sm = s->sweep_ctas;
  s->hist_grid = s->sm_count * per_sm;
  s->lag_shape = s->sweep_shape;
  s->lag_grid = s->hist_grid;
  if (s->fp32() && s->N <= kFusedMaxN) {
    s->lag_grid = s->sm_count;
    if (s->sweep_shape == 3 || s->sweep_shape == 4) {
      s->lag_shape = 4;
      s->lag_grid = 2 * s->sm_count;
    }
  }
  if (s->lag_ctas > 0) {
    // set by the autotuner: as many CTAs per SM as timed fastest beside the passes
    const int lim = s->fp32() ? sweep_blocks_per_sm<float>(s->lag_shape, gen)
                              : sweep_blocks_per_sm<double>(s->lag_shape, false);
    s->lag_grid = s->sm_count * std::max(1, std::min(s->lag_ctas, lim));
  }
  s->f64.sweep_shape = s->f32.sweep_shape = s->sweep_shape;
  s->f64.lag_shape = s->f32.lag_shape = s->lag_shape;
}

template <class R>
void fill_dev(sbiem_s* s, DevFault<R>& f) {
  f.N = s->N;
  f.nmodes = s->nmodes;
  f.L = s->L;
  f.S = s->S;
  f.mu = s->p.mu;
  f.eta = s->eta;
  f.reta = 1.0 / s->eta;
  f.dt_min = s->dt_min;
  f.f0 = s->p.f0;
  f.V0 = s->p.V0;
  f.lnV0 = std::log(s->p.V0);
  f.state_law = s->p.state_law;
  f.newton_epw = 32;  // elements per Newton warp: 32 measured fastest on GB300
  f.spin_limit = s->spin_limit;
  f.newton_maxit = s->p.newton_maxit;
  f.sweep_shape = s->sweep_shape;
  f.lag_shape = s->lag_shape;
  f.newton_tol = s->p.newton_tol;
}

template <class R>
int setup_device(sbiem_s* s, DevFault<R>& f, const DevFault<double>& base) {
  // element and spectral arrays are shared with the FP64 view
  f = DevFault<R>{};
  fill_dev(s, f);
#define COPYP(x) f.x = base.x
  COPYP(V); COPYP(psi); COPYP(th); COPYP(th2); COPYP(thd); COPYP(delta); COPYP(V1); COPYP(thd1); COPYP(Vbar);
  COPYP(V2); COPYP(psi2); COPYP(thd2); COPYP(delta2); COPYP(a); COPYP(b); COPYP(Dc);
  COPYP(xV); COPYP(x1); COPYP(x2); COPYP(lvd); COPYP(rDc);
  COPYP(sig0); COPYP(tau0); COPYP(taur); COPYP(Vp); COPYP(kappa); COPYP(presc);
  COPYP(dhat); COPYP(khat); COPYP(U2); COPYP(Q2); COPYP(AT); COPYP(AN); COPYP(BT); COPYP(BN); COPYP(partial);
  COPYP(counter); COPYP(ring_off); COPYP(w_off); COPYP(Rn); COPYP(Mn); COPYP(head);
  COPYP(chunks); COPYP(nchunks); COPYP(mfirst); COPYP(mcount); COPYP(status); COPYP(steps_done); COPYP(t);
  COPYP(it_sum); COPYP(it_max); COPYP(it_total); COPYP(work); COPYP(w0pow); COPYP(c0pow); COPYP(dhat32); COPYP(khat32);
  COPYP(AT32); COPYP(AN32);
#undef COPYP
  bool ok = true;
  f.ring = alloc_n<Slot<R>>(s, static_cast<size_t>(std::max<int64_t>(s->total_slots, 1)), &ok);
  // two spare entries: the sweep's 16-byte aligned weight copies may read one past the end
  f.w = alloc_n<W2<R>>(s, static_cast<size_t>(s->total_w + 2), &ok);
  f.zt = alloc_n<Cx<R>>(s, s->N, &ok);
  f.Z = alloc_n<Cx<R>>(s, s->N, &ok);
  f.y = alloc_n<Cx<R>>(s, s->N, &ok);
  if (!ok) return nomem(s, "history rings / weights");
  if constexpr (sizeof(R) == 4) {
    // the precision form's passes: Vbar + i kappa Vbar prepared in FP32 by
    // the commit and the pass-1 Newton, U and Q of the step kept in FP32
    f.zin1 = alloc_n<float2>(s, s->N, &ok);
    f.zin2 = alloc_n<float2>(s, s->N, &ok);
    f.U2f = alloc_n<float2>(s, s->nmodes, &ok);
    f.Q2f = alloc_n<float2>(s, s->nmodes, &ok);
  }
  if (!ok) return nomem(s, "FP32 pass buffers");
  f.g = make_geom(s->N, sizeof(Cx<R>));
  if constexpr (sizeof(R) == 8) f.tw = s->tw64;
  else f.tw = s->tw32;
  configure_kernels<R>(f.g);
  return SBIEM_OK;
}

void probe_mark(sbiem_s* s, int k, cudaStream_t st) {
  if (s->pslots) cudaEventRecordWithFlags(s->pev[4 * s->pcur + k], st, cudaEventRecordExternal);
}

template <class R>
void enqueue_step_t(sbiem_s* s, const DevFault<R>& f, int m, cudaStream_t st) {
  probe_mark(s, 0, st);
  probe_mark(s, 1, st);
  launch_history<R>(f, m, s->hist_grid, st);
  probe_mark(s, 2, st);
  launch_pass<R>(f, 1, m, st);
  launch_pass<R>(f, 2, m, st);
  if (m > 1) launch_push_multi<R>(f, m, st);
  launch_commit<R>(f, m, st);
  probe_mark(s, 3, st);
}

// Overlapped step of m = 2^p dt_min: AT/AN already hold this step's sums;
// the side branch sweeps the history for the next step (weights shifted by
// 2m, into BT/BN) while the passes run; the commit adds this step's slot.
template <class R>
void enqueue_step_lag_t(sbiem_s* s, const DevFault<R>& f, int m, cudaStream_t st) {
  int p = 0;
  while ((1 << p) < m) ++p;
  cudaEventRecord(s->ev_fork, st);
  // the side branch's sweep is dispatched once every CTA of the pass-1
  // spectral kernel has started (a programmatic event): when the sweep was
  // dispatched first it could hold the SMs the pass needed, and which of
  // the graph's two branches reached the GPU first changed from one graph
  // instance to the next (flushed N = 4096 steps of 41 or 51 us by
  // instance; 41 us every time in this order)
  launch_spectral<R>(f, 1, m, st, s->ev_started);
  cudaStreamWaitEvent(s->side, s->ev_fork, 0);
  cudaStreamWaitEvent(s->side, s->ev_started, 0);
  launch_history_ahead<R>(f, m, s->lag_grid, s->side);
  cudaEventRecord(s->ev_join, s->side);
  launch_newton<R>(f, 1, m, st);
  launch_pass<R>(f, 2, m, st);
  cudaStreamWaitEvent(st, s->ev_join, 0);
  if (m > 1) launch_push_multi<R>(f, m, st);
  launch_commit<R>(f, m, st, p);
}

// The step without its commit: pass-2 results stay staged (delta2, V2, ...).
template <class R>
void enqueue_trial_t(sbiem_s* s, const DevFault<R>& f, int m, cudaStream_t st) {
  launch_history<R>(f, m, s->hist_grid, st);
  launch_pass<R>(f, 1, m, st);
  launch_pass<R>(f, 2, m, st);
}

void enqueue_step(sbiem_s* s, int m, cudaStream_t st) {
  if (s->fp32()) enqueue_step_t<float>(s, s->f32, m, st);
  else enqueue_step_t<double>(s, s->f64, m, st);
}

void enqueue_trial(sbiem_s* s, int m, cudaStream_t st) {
  if (s->fp32()) enqueue_trial_t<float>(s, s->f32, m, st);
  else enqueue_trial_t<double>(s, s->f64, m, st);
}

void ring_undo(sbiem_s* s, int m, int dir) {
  if (s->fp32()) launch_ring_undo<float>(s->f32, m, s->undo, dir, s->stream);
  else launch_ring_undo<double>(s->f64, m, s->undo, dir, s->stream);
}

// Device buffers of the state snapshot (allocated on first use).
bool ensure_snapshot(sbiem_s* s) {
  bool ok = true;
  if (!s->snap) {
    s->snap = alloc_n<double>(s, static_cast<size_t>(6) * s->N + 1, &ok);
    s->snap_spec = alloc_n<double2>(s, static_cast<size_t>(2) * s->nmodes, &ok);
    s->snap_head = alloc_n<int32_t>(s, s->nmodes, &ok);
    s->snap_steps = alloc_n<long long>(s, 1, &ok);
  }
  return ok && s->snap && s->snap_spec && s->snap_head && s->snap_steps;
}

// Save (save = true) or restore the committed state that a step changes.
int snapshot(sbiem_s* s, bool save) {
  auto& f = s->f64;
  const size_t nb = sizeof(double) * s->N;
  double* arrs[] = {f.V, f.xV, f.psi, f.thd, f.delta, f.th};
  for (int k = 0; k < 6; ++k) {
    double* sn = s->snap + static_cast<size_t>(k) * s->N;
    CK(cudaMemcpyAsync(save ? sn : arrs[k], save ? arrs[k] : sn, nb, cudaMemcpyDeviceToDevice, s->stream));
  }
  double* snt = s->snap + static_cast<size_t>(6) * s->N;
  CK(cudaMemcpyAsync(save ? snt : f.t, save ? f.t : snt, sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  const size_t sb = sizeof(double2) * s->nmodes;
  CK(cudaMemcpyAsync(save ? s->snap_spec : f.dhat, save ? f.dhat : s->snap_spec, sb, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(save ? s->snap_spec + s->nmodes : f.khat, save ? f.khat : s->snap_spec + s->nmodes, sb,
                     cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(save ? s->snap_head : f.head, save ? f.head : s->snap_head, sizeof(int32_t) * s->nmodes,
                     cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(save ? s->snap_steps : f.steps_done, save ? f.steps_done : s->snap_steps, sizeof(long long),
                     cudaMemcpyDeviceToDevice, s->stream));
  if (!save && f.dhat32) {
    // the FP32 copies of the restored running sums
    launch_to_float2(f.dhat, f.dhat32, s->nmodes, s->stream);
    launch_to_float2(f.khat, f.khat32, s->nmodes, s->stream);
  }
  if (!save && s->f32.zin1) launch_zin(f.V, f.kappa, s->f32.zin1, s->N, s->stream);
  return SBIEM_OK;
}

int status_to_code(unsigned st) {
  if (st & SBIEM_FLAG_NEWTON) return SBIEM_ERR_NEWTON;
  if (st & SBIEM_FLAG_OPENING) return SBIEM_ERR_OPENING;
  if (st & SBIEM_FLAG_STATE) return SBIEM_ERR_STATE;
  if (st & SBIEM_FLAG_WAIT) return SBIEM_ERR_WAIT;
  return SBIEM_OK;
}

int dt_to_m(const sbiem_s* s, double dt, int* m) {
  if (!(dt > 0.0)) return fail(SBIEM_ERR_INVALID, "dt must be positive");
  const double r = dt / s->dt_min;
  const double mr = std::floor(r + 0.5);
  if (mr < 1.0 || std::fabs(r - mr) > 1e-9 * mr || mr > 1e9)
    return fail(SBIEM_ERR_INVALID, "dt must be an integer multiple m >= 1 of dt_min = beta_min dx / cs");
  *m = static_cast<int>(mr);
  return SBIEM_OK;
}

// F[delta], F[kappa delta] of the committed slip (FP64 utility FFT).
int recompute_spectral_sums(sbiem_s* s) {
  auto& f = s->f64;
  launch_pack(s->N, f.delta, f.delta, f.kappa, s->u_a, s->stream);
  launch_fft64(s->g64, s->tw64, s->u_a, s->u_b, s->u_c, false, s->stream);
  launch_unpack(s->N, s->u_c, f.dhat, f.khat, s->stream);
  if (f.dhat32) {
    launch_to_float2(f.dhat, f.dhat32, s->nmodes, s->stream);
    launch_to_float2(f.khat, f.khat32, s->nmodes, s->stream);
  }
  if (s->f32.zin1) launch_zin(f.V, f.kappa, s->f32.zin1, s->N, s->stream);
  CK(cudaGetLastError());
  return SBIEM_OK;
}

}  // namespace

extern "C" {

void sbiem_default_params(sbiem_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->beta_min = 0.25;
  p->eta_w = 1.0;
  p->kc_L = 200.0;
  p->kcN_L = 0.0;
  p->kc_units = 0;
  p->precision = 0;
  p->state_law = 0;
  p->newton_maxit = 50;
  p->newton_tol = 1e-12;
}

const char* sbiem_strerror(int code) {
  switch (code) {
    case SBIEM_OK: return "ok";
    case SBIEM_ERR_INVALID: return "invalid argument";
    case SBIEM_ERR_NOMEM: return "device out of memory";
    case SBIEM_ERR_CUDA: return "CUDA runtime error";
    case SBIEM_ERR_NEWTON: return "friction Newton iteration did not converge";
    case SBIEM_ERR_OPENING: return "effective normal stress not positive (fault opening)";
    case SBIEM_ERR_STATE: return "state variable not positive";
    case SBIEM_ERR_DTMIN: return "failure at the minimum time step";
    case SBIEM_ERR_UNSUPPORTED: return "unsupported request";
    case SBIEM_ERR_WAIT: return "a device-side wait ran past its limit";
    default: return "unknown error";
  }
}

const char* sbiem_last_error(void) { return g_last_error.c_str(); }

int sbiem_create(sbiem_t* out, const sbiem_params* pin, const double* h, const double* kappa,
                 const double* a, const double* b, const double* Dc, const double* sigma_load,
                 const double* tau_load, const double* tau_load_rate, const uint8_t* prescribed,
                 const double* V_presc, const double* V_init, const double* theta_init) {
  if (!out || !pin) return fail(SBIEM_ERR_INVALID, "NULL handle or parameter pointer");
  *out = nullptr;
  const sbiem_params& p = *pin;
  if (!is_pow2(p.N) || p.N < 16 || p.N > (1 << 20))
    return fail(SBIEM_ERR_INVALID, "N must be a power of two in [16, 2^20]");
  if (!(p.dx > 0) || !(p.mu > 0) || !(p.cs > 0) || !(p.cp > p.cs) || !(p.beta_min > 0) ||
      !(p.eta_w >= 0) || !(p.kc_L > 0) || !(p.kcN_L >= 0) || !(p.V0 > 0) || !(p.newton_tol > 0) || p.newton_maxit < 1)
    return fail(SBIEM_ERR_INVALID,
                "parameters out of range (dx, mu, cs < cp, beta_min, eta_w, kc_L, kcN_L, V0, Newton)");
  if (p.precision != 0 && p.precision != 1) return fail(SBIEM_ERR_INVALID, "precision must be 0 or 1");
  if (p.state_law != 0 && p.state_law != 1) return fail(SBIEM_ERR_INVALID, "state_law must be 0 or 1");
  if (p.kc_units != 0 && p.kc_units != 1) return fail(SBIEM_ERR_INVALID, "kc_units must be 0 or 1");
  if (p.quadrature != 0 && p.quadrature != 1) return fail(SBIEM_ERR_INVALID, "quadrature must be 0 or 1");
  if ((!h && !kappa) || !a || !b || !Dc || !sigma_load || !V_init || !theta_init)
    return fail(SBIEM_ERR_INVALID, "required input array is NULL");
  if (prescribed && !V_presc) return fail(SBIEM_ERR_INVALID, "prescribed given without V_presc");
  const int N = static_cast<int>(p.N);
  for (int i = 0; i < N; ++i) {
    const bool pr = prescribed && prescribed[i];
    if (!(Dc[i] > 0) || !(sigma_load[i] > 0) || !(theta_init[i] > 0))
      return fail(SBIEM_ERR_INVALID, "Dc, sigma_load and theta_init must be positive at element " + std::to_string(i));
    if (!pr && (!(a[i] > 0) || !(V_init[i] > 0)))
      return fail(SBIEM_ERR_INVALID, "a and V_init must be positive on frictional element " + std::to_string(i));
  }

  auto* s = new sbiem_s();
  s->p = p;
  cudaGetDevice(&s->device);
  cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  if (cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_started, cudaEventDisableTiming) != cudaSuccess) {
    free_all(s);
    delete s;
    return fail(SBIEM_ERR_CUDA, "stream / event creation failed");
  }
  s->stream = s->own;
  s->N = N;
  s->nmodes = N / 2 + 1;
  s->L = N * p.dx;
  s->dt_min = p.beta_min * p.dx / p.cs;
  const double r = p.cs / p.cp;
  s->S = p.mu * (1.0 - r * r);
  s->eta = p.mu / (2.0 * p.cs);
  windows(p, s->L, s->dt_min, s->M, s->MT, s->MN);
  {
    // bulk-async sweep: chunks of one stage buffer (512 lags FP32, 256 FP64),
    // every resident CTA streaming; the overlapped sweep keeps one CTA per SM
    // so the pass kernels find room beside it
    if (s->fp32()) configure_kernels<float>(make_geom(N, sizeof(float2)));
    else configure_kernels<double>(make_geom(N, sizeof(double2)));
    s->sweep_shape = kDefaultSweepShape;
    sweep_config(s);  // grids again below once the weight form is known
    s->chunk_slots = sweep_chunk_slots(p.precision, s->sweep_shape);
  }
  s->Rn.assign(s->nmodes, 0);
  s->ring_off.assign(s->nmodes + 1, 0);
  s->w_off.assign(s->nmodes + 1, 0);
  for (int n = 0; n < s->nmodes; ++n) {
    s->Rn[n] = std::max<int64_t>(s->M[n] - 1, 0);
    s->ring_off[n + 1] = s->ring_off[n] + s->Rn[n];
    s->w_off[n + 1] = s->w_off[n] + s->M[n];
    const int64_t cs = s->chunk_slots;
    const int64_t cnt = (s->Rn[n] + cs - 1) / cs;
    for (int64_t c = 0; c < cnt; ++c) {
      Chunk ch{};
      ch.mode = n;
      ch.first = static_cast<int32_t>(s->chunks.size() - c);
      ch.count = static_cast<int32_t>(cnt);
      ch.i0 = c * cs;
      ch.i1 = std::min<int64_t>((c + 1) * cs, s->Rn[n]);
      s->chunks.push_back(ch);
    }
  }
  // fix 'first': index of the mode's first chunk
  for (size_t c = 0; c < s->chunks.size();) {
    const int cnt = s->chunks[c].count;
    for (int q = 0; q < cnt; ++q) s->chunks[c + q].first = static_cast<int32_t>(c);
    c += cnt;
  }
  std::vector<int32_t> mfirst(s->nmodes, 0), mcount(s->nmodes, 0);
  for (size_t c = 0; c < s->chunks.size(); ++c) {
    const int n = s->chunks[c].mode;
    if (mcount[n] == 0) mfirst[n] = static_cast<int32_t>(c);
    ++mcount[n];
  }
  s->total_slots = s->ring_off[s->nmodes];
  s->total_w = s->w_off[s->nmodes];
  s->planned_ring = s->total_slots * (s->fp32() ? 16 : 32);
  s->planned_w = (s->total_w + 2) * (s->fp32() ? 8 : 16);
  s->planned_bytes = s->planned_ring + s->planned_w + static_cast<int64_t>(s->chunks.size()) * 56 +
                     static_cast<int64_t>(N) * 8 * 40 + static_cast<int64_t>(s->nmodes) * 16 * (20 + kPow2Slots);
  if (s->total_slots > (int64_t(1) << 31) || s->Rn[1] > (int64_t(1) << 30)) {
    free_all(s);
    delete s;
    return fail(SBIEM_ERR_INVALID, "history too long for this build");
  }

  auto& f = s->f64;
  fill_dev(s, f);
  bool ok = true;
  double** darr[] = {&f.V, &f.psi, &f.thd, &f.delta, &f.V1, &f.thd1, &f.Vbar, &f.V2, &f.psi2, &f.thd2,
                     &f.delta2, &f.a, &f.b, &f.Dc, &f.sig0, &f.tau0, &f.taur, &f.Vp, &f.kappa,
                     &f.xV, &f.x1, &f.x2, &f.lvd, &f.th, &f.th2, &f.rDc};
  for (double** d : darr) *d = alloc_n<double>(s, N, &ok);
  f.presc = alloc_n<uint8_t>(s, N, &ok);
  double2** carr[] = {&f.dhat, &f.khat, &f.U2, &f.Q2, &f.AT, &f.AN, &f.BT, &f.BN};
  for (double2** c : carr) *c = alloc_n<double2>(s, s->nmodes, &ok);
  f.partial = alloc_n<double4>(s, std::max<size_t>(s->chunks.size(), 1), &ok);
  f.w0pow = alloc_n<double2>(s, static_cast<size_t>(s->nmodes) * kPow2Slots, &ok);
  if (s->fp32()) {
    f.c0pow = alloc_n<float2>(s, static_cast<size_t>(s->nmodes) * kPow2Slots, &ok);
    f.dhat32 = alloc_n<float2>(s, s->nmodes, &ok);
    f.khat32 = alloc_n<float2>(s, s->nmodes, &ok);
    f.AT32 = alloc_n<float2>(s, s->nmodes, &ok);
    f.AN32 = alloc_n<float2>(s, s->nmodes, &ok);
  }
  f.counter = alloc_n<int>(s, s->nmodes, &ok);
  int64_t* d_roff = alloc_n<int64_t>(s, s->nmodes + 1, &ok);
  int64_t* d_woff = alloc_n<int64_t>(s, s->nmodes + 1, &ok);
  int32_t* d_Rn = alloc_n<int32_t>(s, s->nmodes, &ok);
  int32_t* d_Mn = alloc_n<int32_t>(s, s->nmodes, &ok);
  f.head = alloc_n<int32_t>(s, s->nmodes, &ok);
  Chunk* d_chunks = alloc_n<Chunk>(s, std::max<size_t>(s->chunks.size(), 1), &ok);
  int32_t* d_mfirst = alloc_n<int32_t>(s, s->nmodes, &ok);
  int32_t* d_mcount = alloc_n<int32_t>(s, s->nmodes, &ok);
  f.status = alloc_n<unsigned>(s, 1, &ok);
  f.steps_done = alloc_n<long long>(s, 1, &ok);
  f.t = alloc_n<double>(s, 1, &ok);
  f.it_sum = alloc_n<unsigned long long>(s, 1, &ok);
  f.work = alloc_n<int>(s, 1, &ok);
  f.it_max = alloc_n<int>(s, 1, &ok);
  f.it_total = alloc_n<unsigned long long>(s, 2, &ok);
  s->tw64 = alloc_n<double2>(s, N, &ok);
  s->u_a = alloc_n<double2>(s, N, &ok);
  s->u_b = alloc_n<double2>(s, N, &ok);
  s->u_c = alloc_n<double2>(s, N, &ok);
  if (s->fp32()) s->tw32 = alloc_n<float2>(s, N, &ok);
  f.ring_off = d_roff;
  f.w_off = d_woff;
  f.Rn = d_Rn;
  f.Mn = d_Mn;
  f.chunks = d_chunks;
  f.nchunks = static_cast<int>(s->chunks.size());
  f.mfirst = d_mfirst;
  f.mcount = d_mcount;
  if (!ok) {
    const int rc_nm = nomem(s, "element and spectral arrays");
    free_all(s);
    delete s;
    return rc_nm;
  }
  cudaMallocHost(&s->h_status, sizeof(unsigned));
  cudaMallocHost(&s->h_steps, sizeof(long long));

  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream);
  };
  std::vector<int32_t> Rn32(s->nmodes), Mn32(s->nmodes);
  for (int n = 0; n < s->nmodes; ++n) {
    Rn32[n] = static_cast<int32_t>(s->Rn[n]);
    Mn32[n] = static_cast<int32_t>(s->M[n]);
  }
  std::vector<double> tw;
  build_twiddles(N, tw);
  std::vector<float> tw32;
  if (s->fp32()) {
    tw32.resize(tw.size());
    for (size_t i = 0; i < tw.size(); ++i) tw32[i] = static_cast<float>(tw[i]);
  }
  // friction arrays, load, state
  std::vector<double> psi(N), thd(N), taul(N, 0.0), taur(N, 0.0), Vp(N, 0.0), V(N), xV(N), lvd(N), rDc(N);
  std::vector<uint8_t> pr(N, 0);
  for (int i = 0; i < N; ++i) {
    pr[i] = (prescribed && prescribed[i]) ? 1 : 0;
    Vp[i] = pr[i] ? V_presc[i] : 0.0;
    V[i] = pr[i] ? V_presc[i] : V_init[i];
    psi[i] = std::log(theta_init[i]);
    thd[i] = 1.0 - theta_init[i] * V[i] / Dc[i];
    xV[i] = V[i] > 0.0 ? std::log(V[i]) : -745.0;
    lvd[i] = std::log(p.V0 / Dc[i]);
    rDc[i] = 1.0 / Dc[i];
    if (tau_load_rate) taur[i] = tau_load_rate[i];
    if (tau_load) {
      taul[i] = tau_load[i];
    } else if (!pr[i]) {
      // equilibrium with the initial state (Eq. momentum + radiation damping)
      const double fr = p.f0 + a[i] * std::log(V[i] / p.V0) + b[i] * std::log(theta_init[i] * p.V0 / Dc[i]);
      taul[i] = sigma_load[i] * fr + s->eta * V[i];
    }
  }
  const size_t nb = sizeof(double) * N;
  bool cu = up(f.a, a, nb) == cudaSuccess && up(f.b, b, nb) == cudaSuccess && up(f.Dc, Dc, nb) == cudaSuccess &&
            up(f.sig0, sigma_load, nb) == cudaSuccess && up(f.tau0, taul.data(), nb) == cudaSuccess &&
            up(f.taur, taur.data(), nb) == cudaSuccess && up(f.Vp, Vp.data(), nb) == cudaSuccess &&
            up(f.presc, pr.data(), N) == cudaSuccess && up(f.V, V.data(), nb) == cudaSuccess &&
            up(f.psi, psi.data(), nb) == cudaSuccess && up(f.th, theta_init, nb) == cudaSuccess &&
            up(f.thd, thd.data(), nb) == cudaSuccess &&
            up(f.xV, xV.data(), nb) == cudaSuccess && up(f.lvd, lvd.data(), nb) == cudaSuccess &&
            up(f.rDc, rDc.data(), nb) == cudaSuccess &&
            up(d_roff, s->ring_off.data(), sizeof(int64_t) * (s->nmodes + 1)) == cudaSuccess &&
            up(d_woff, s->w_off.data(), sizeof(int64_t) * (s->nmodes + 1)) == cudaSuccess &&
            up(d_Rn, Rn32.data(), sizeof(int32_t) * s->nmodes) == cudaSuccess &&
            up(d_Mn, Mn32.data(), sizeof(int32_t) * s->nmodes) == cudaSuccess &&
            (s->chunks.empty() || up(d_chunks, s->chunks.data(), sizeof(Chunk) * s->chunks.size()) == cudaSuccess) &&
            up(d_mfirst, mfirst.data(), sizeof(int32_t) * s->nmodes) == cudaSuccess &&
            up(d_mcount, mcount.data(), sizeof(int32_t) * s->nmodes) == cudaSuccess &&
            up(s->tw64, tw.data(), sizeof(double) * tw.size()) == cudaSuccess &&
            (!s->fp32() || up(s->tw32, tw32.data(), sizeof(float) * tw32.size()) == cudaSuccess);
  s->g64 = make_geom(N, sizeof(double2));
  configure_kernels<double>(s->g64);
  // curvature: given, or kappa = h'' by spectral differentiation (Sec. 2.2, small slope)
  if (kappa) {
    cu = cu && up(f.kappa, kappa, nb) == cudaSuccess;
  } else {
    cu = cu && up(f.Vbar, h, nb) == cudaSuccess;  // scratch for h
    launch_pack(N, f.Vbar, nullptr, nullptr, s->u_a, s->stream);
    launch_fft64(s->g64, s->tw64, s->u_a, s->u_b, s->u_c, false, s->stream);
    launch_d2(N, s->L, s->u_c, s->stream);
    launch_fft64(s->g64, s->tw64, s->u_c, s->u_b, s->u_a, true, s->stream);
    launch_real_part(N, s->u_a, f.kappa, s->stream);
  }
  // kernel tables: piecewise Chebyshev of C^T, C^N on the s range the weights need
  double smax = 0.0;
  for (int n = 1; n < s->nmodes; ++n) {
    const double k = 2.0 * M_PI * n / s->L;
    smax = std::max(smax, p.cs * k * (s->M[n] - 0.5) * s->dt_min);
  }
  ChebTable tab;
  build_cheb(r, smax + 1.0, &tab);
  double* d_cheb = alloc_n<double>(s, tab.coef.size(), &ok);
  if (!ok || !cu) {
    free_all(s);
    delete s;
    return fail(ok ? SBIEM_ERR_CUDA : SBIEM_ERR_NOMEM, "upload failed");
  }
  up(d_cheb, tab.coef.data(), sizeof(double) * tab.coef.size());
  // the two kernels' own windows, when they differ (two cutting planes)
  int32_t* d_MT = nullptr;
  int32_t* d_MN = nullptr;
  if (s->MT != s->MN) {
    std::vector<int32_t> mt(s->nmodes), mn(s->nmodes);
    for (int n = 0; n < s->nmodes; ++n) {
      mt[n] = static_cast<int32_t>(s->MT[n]);
      mn[n] = static_cast<int32_t>(s->MN[n]);
    }
    d_MT = alloc_n<int32_t>(s, s->nmodes, &ok);
    d_MN = alloc_n<int32_t>(s, s->nmodes, &ok);
    if (!ok || up(d_MT, mt.data(), sizeof(int32_t) * s->nmodes) != cudaSuccess ||
        up(d_MN, mn.data(), sizeof(int32_t) * s->nmodes) != cudaSuccess) {
      free_all(s);
      delete s;
      return fail(SBIEM_ERR_NOMEM, "upload failed (windows)");
    }
  }
  int rc;
  if (s->fp32()) {
    rc = setup_device<float>(s, s->f32, f);
    if (rc == SBIEM_OK) {
      launch_weights<float>(s->f32, d_cheb, tab.npieces, tab.deg, tab.h, p.cs, d_MT, d_MN, p.quadrature,
                            s->stream);
      launch_weight_pow2<float>(s->f32, s->stream);
    }
    // the sweep's on-chip weights: the table of dt C(s) over the s range of
    // the windows, and per mode ds = c_s k_n dt_min (two floats) with the
    // two fields' windows; kept only while the table fits beside the stages
    std::vector<float> gtab;
    int gp = 0;
    double gerr = 0.0;
    build_gen_table(r, s->dt_min, smax, gtab, &gp, &gerr);
    if (rc == SBIEM_OK && p.quadrature == 0 &&
        static_cast<int64_t>(gp) * (kGenDeg + 1) * 8 <= kGenMaxTableBytes) {
      std::vector<float4> wg(s->nmodes);
      for (int n = 0; n < s->nmodes; ++n) {
        const double ds = p.cs * (2.0 * M_PI * n / s->L) * s->dt_min;
        const float hi = static_cast<float>(ds);
        const float lo = static_cast<float>(ds - static_cast<double>(hi));
        int32_t mt = static_cast<int32_t>(s->MT[n]), mn = static_cast<int32_t>(s->MN[n]);
        float fmt, fmn;
        std::memcpy(&fmt, &mt, 4);
        std::memcpy(&fmn, &mn, 4);
        wg[n] = make_float4(hi, lo, fmt, fmn);
      }
      float4* d_wtab = alloc_n<float4>(s, gtab.size() / 4, &ok);
      float4* d_wgen = alloc_n<float4>(s, s->nmodes, &ok);
      if (!ok || up(d_wtab, gtab.data(), sizeof(float) * gtab.size()) != cudaSuccess ||
          up(d_wgen, wg.data(), sizeof(float4) * s->nmodes) != cudaSuccess) {
        rc = nomem(s, "weight table");
      } else {
        s->f32.wtab = d_wtab;
        s->f32.wgen = d_wgen;
        s->f32.wtab_pieces = gp;
        s->gen_pieces = gp;
        s->gen_err = gerr;
        s->gen_ds_max = kGenDsMaxDefault;
      }
    }
    sweep_config(s);
  } else {
    f.ring = alloc_n<Slot64>(s, static_cast<size_t>(std::max<int64_t>(s->total_slots, 1)), &ok);
    f.w = alloc_n<W2<double>>(s, static_cast<size_t>(s->total_w + 2), &ok);
    f.zt = alloc_n<double2>(s, N, &ok);
    f.Z = alloc_n<double2>(s, N, &ok);
    f.y = alloc_n<double2>(s, N, &ok);
    f.g = make_geom(N, sizeof(double2));
    f.tw = s->tw64;
    rc = ok ? SBIEM_OK : nomem(s, "history rings / weights");
    if (rc == SBIEM_OK) {
      launch_weights<double>(f, d_cheb, tab.npieces, tab.deg, tab.h, p.cs, d_MT, d_MN, p.quadrature, s->stream);
      launch_weight_pow2<double>(f, s->stream);
    }
  }
  if (rc == SBIEM_OK) rc = recompute_spectral_sums(s);
  if (rc == SBIEM_OK && cudaStreamSynchronize(s->stream) != cudaSuccess)
    rc = fail(SBIEM_ERR_CUDA, std::string("create: ") + cudaGetErrorString(cudaGetLastError()));
  if (rc != SBIEM_OK) {
    free_all(s);
    delete s;
    return rc;
  }
  *out = s;
  return SBIEM_OK;
}

void sbiem_destroy(sbiem_t s) {
  if (!s) return;
  free_all(s);
  delete s;
}

int sbiem_set_stream(sbiem_t s, void* stream) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  CK(cudaStreamSynchronize(s->stream));
  // NULL is the legacy default stream (cudaStreamLegacy), ordered with other
  // work on it; step graphs are still captured on the handle's own stream
  s->stream = stream ? static_cast<cudaStream_t>(stream) : cudaStreamLegacy;
  s->user_stream = true;
  return SBIEM_OK;
}

int sbiem_status(sbiem_t s, uint32_t* flags, int64_t* steps_done, int clear) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  CK(cudaMemcpyAsync(s->h_status, s->f64.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(s->h_steps, s->f64.steps_done, sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (flags) *flags = *s->h_status;
  if (steps_done) *steps_done = *s->h_steps;
  if (*s->h_status) s->lag_m = -1;  // a rejected step left AT/AN of its start
  if (clear) CK(cudaMemsetAsync(s->f64.status, 0, sizeof(unsigned), s->stream));
  return SBIEM_OK;
}

}  // extern "C"

namespace {

// The overlapped step graph of m dt_min (captured and instantiated once).
int lag_graph(sbiem_s* s, int m) {
  if (s->lag_graphs.count(m)) return SBIEM_OK;
  cudaGraph_t gdef = nullptr;
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaStreamBeginCapture(s->own, cudaStreamCaptureModeThreadLocal));
  if (s->fp32()) enqueue_step_lag_t<float>(s, s->f32, m, s->own);
  else enqueue_step_lag_t<double>(s, s->f64, m, s->own);
  cudaError_t e1 = cudaGetLastError();
  cudaError_t e2 = cudaStreamEndCapture(s->own, &gdef);
  if (e1 != cudaSuccess || e2 != cudaSuccess)
    return fail(SBIEM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
  cudaGraphExec_t exec = nullptr;
  CK(cudaGraphInstantiate(&exec, gdef, 0));
  s->lag_graphs[m] = exec;
  s->lag_defs[m] = gdef;
  return SBIEM_OK;
}

}  // namespace

extern "C" {

int sbiem_step_kernels(sbiem_t s, double dt, int64_t* kernels) {
  if (!s || !kernels) return fail(SBIEM_ERR_INVALID, "NULL argument");
  int m;
  int rc = dt_to_m(s, dt, &m);
  if (rc) return rc;
  if (!is_pow2(m) || m > (1 << 30)) return fail(SBIEM_ERR_INVALID, "m must be a power of two");
  rc = lag_graph(s, m);
  if (rc) return rc;
  cudaGraph_t gdef = s->lag_defs[m];
  size_t nn = 0;
  CK(cudaGraphGetNodes(gdef, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CK(cudaGraphGetNodes(gdef, nodes.data(), &nn));
  int64_t k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    CK(cudaGraphNodeGetType(nd, &ty));
    if (ty == cudaGraphNodeTypeKernel) ++k;
  }
  *kernels = k;
  return SBIEM_OK;
}

int sbiem_step(sbiem_t s, double dt) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  int m;
  int rc = dt_to_m(s, dt, &m);
  if (rc) return rc;
  uint32_t before;
  rc = sbiem_status(s, &before, nullptr, 1);
  if (rc) return rc;
  if (s->pslots) s->pcur = static_cast<int>(s->pcount++ % s->pslots);
  s->lag_m = -1;
  enqueue_step(s, m, s->stream);
  CK(cudaGetLastError());
  uint32_t st;
  rc = sbiem_status(s, &st, nullptr, 1);
  if (rc) return rc;
  rc = status_to_code(st);
  if (rc) return fail(rc, "step rejected; state left at the start of the step");
  return SBIEM_OK;
}

int sbiem_enqueue(sbiem_t s, double dt, int64_t nsteps) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  if (nsteps < 0) return fail(SBIEM_ERR_INVALID, "nsteps < 0");
  int m;
  int rc = dt_to_m(s, dt, &m);
  if (rc) return rc;
  if (nsteps == 0) return SBIEM_OK;
  if (s->pslots == 0 && is_pow2(m) && m <= (1 << 30)) {
    // overlapped form (steps of 2^p dt_min, no timing probe)
    rc = lag_graph(s, m);
    if (rc) return rc;
    auto lt = s->lag_graphs.find(m);
    if (s->lag_m != m) {
      // prologue: this step's full sums
      if (s->fp32()) launch_history<float>(s->f32, m, s->hist_grid, s->stream);
      else launch_history<double>(s->f64, m, s->hist_grid, s->stream);
      CK(cudaGetLastError());
    }
    for (int64_t k = 0; k < nsteps; ++k) CK(cudaGraphLaunch(lt->second, s->stream));
    s->lag_m = m;
    return SBIEM_OK;
  }
  s->lag_m = -1;
  auto it = s->graphs.find(m);
  if (it == s->graphs.end()) {
    // capture one step on the handle's own stream, replay it on s->stream
    cudaGraph_t gdef = nullptr;
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaStreamBeginCapture(s->own, cudaStreamCaptureModeThreadLocal));
    s->pcur = 0;
    enqueue_step(s, m, s->own);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamEndCapture(s->own, &gdef);
    if (e1 != cudaSuccess || e2 != cudaSuccess)
      return fail(SBIEM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    cudaGraphExec_t exec = nullptr;
    CK(cudaGraphInstantiate(&exec, gdef, 0));
    s->graphs[m] = exec;
    s->graph_defs[m] = gdef;
    if (s->pslots) {
      // the event-record nodes of the probe marks, in mark order
      size_t nn = 0;
      CK(cudaGraphGetNodes(gdef, nullptr, &nn));
      std::vector<cudaGraphNode_t> nodes(nn);
      CK(cudaGraphGetNodes(gdef, nodes.data(), &nn));
      std::vector<cudaGraphNode_t> marks(4, nullptr);
      for (auto nd : nodes) {
        cudaGraphNodeType ty;
        CK(cudaGraphNodeGetType(nd, &ty));
        if (ty != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t e;
        CK(cudaGraphEventRecordNodeGetEvent(nd, &e));
        for (int k = 0; k < 4; ++k)
          if (e == s->pev[k]) marks[k] = nd;
      }
      for (auto nd : marks)
        if (!nd) return fail(SBIEM_ERR_CUDA, "probe event nodes not found in the step graph");
      s->pnodes[m] = marks;
    }
    it = s->graphs.find(m);
  }
  for (int64_t k = 0; k < nsteps; ++k) {
    if (s->pslots > 1) {
      const int slot = static_cast<int>(s->pcount++ % s->pslots);
      const auto& marks = s->pnodes[m];
      for (int q = 0; q < 4; ++q)
        CK(cudaGraphExecEventRecordNodeSetEvent(it->second, marks[q], s->pev[4 * slot + q]));
    }
    CK(cudaGraphLaunch(it->second, s->stream));
  }
  return SBIEM_OK;
}

}  // extern "C"

namespace {

// After accepted step `accepted` of sbiem_run: the output callback, when one
// is set and the step is a multiple of its period (or the run's last).
// *stop is set when the callback asks to stop.
int run_output(sbiem_s* s, int64_t accepted, double t, int64_t m, bool last, bool* stop) {
  if (!s->out_cb || accepted == 0) return SBIEM_OK;
  if (!last && accepted % s->out_every != 0) return SBIEM_OK;
  const size_t nb = sizeof(double) * s->N;
  CK(cudaMemcpyAsync(s->h_out, s->f64.delta, nb, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(s->h_out + s->N, s->f64.V, nb, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (s->out_cb(s->out_user, accepted, t, m, s->h_out, s->h_out + s->N, s->N) != 0) *stop = true;
  return SBIEM_OK;
}

}  // namespace

extern "C" {

int sbiem_set_output(sbiem_t s, sbiem_output_fn cb, void* user, int64_t every) {
  if (!s || (cb && every < 1)) return fail(SBIEM_ERR_INVALID, "NULL handle or every < 1");
  if (cb && !s->h_out && cudaMallocHost(&s->h_out, sizeof(double) * 2 * s->N) != cudaSuccess)
    return fail(SBIEM_ERR_NOMEM, "page-locked output buffers");
  s->out_cb = cb;
  s->out_user = user;
  s->out_every = cb ? every : 0;
  return SBIEM_OK;
}

int sbiem_run(sbiem_t s, double t_end, double eps0, int64_t m0, int64_t m_max, int64_t max_steps,
              int64_t* steps_out, int64_t* m_next, double* t_out, int64_t* m_hist) {
  if (!s || !(eps0 > 0) || m0 < 1 || m_max < 1 || max_steps < 0) return fail(SBIEM_ERR_INVALID, "bad argument");
  s->lag_m = -1;  // trial steps and rollbacks below compute their own sums
  auto& f = s->f64;
  bool ok = ensure_snapshot(s);
  if (!s->undo) {
    s->dfull = alloc_n<double>(s, s->N, &ok);
    s->d_err = alloc_n<double>(s, 1, &ok);
    const size_t slot = s->fp32() ? sizeof(Slot32) : sizeof(Slot64);
    s->undo = dev_alloc(s, slot * static_cast<size_t>(std::max<int64_t>(s->total_slots, 1)));
    if (!s->undo) ok = false;
  }
  if (!ok) return fail(SBIEM_ERR_NOMEM, "adaptive run: snapshot allocation failed");
  // m: a power of two in [1, 2^30]
  auto pow2_floor = [](int64_t v) {
    int64_t p = 1;
    while (p * 2 <= v && p < (int64_t(1) << 30)) p *= 2;
    return p;
  };
  int64_t m = pow2_floor(m0);
  m_max = pow2_floor(m_max);
  double t = 0.0;
  CK(cudaMemcpyAsync(&t, f.t, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  int64_t accepted = 0;
  uint32_t st = 0;
  int rc = SBIEM_OK;
  while (t < t_end * (1.0 - 1e-15) && accepted < max_steps) {
    if (m == 1) {
      enqueue_step(s, 1, s->stream);
      rc = sbiem_status(s, &st, nullptr, 1);
      if (rc) return rc;
      if (st) {
        rc = fail(SBIEM_ERR_DTMIN, "step failed at dt_min (status bits " + std::to_string(st) +
                                       "); state left at the start of the step");
        break;
      }
      if (m_hist) m_hist[accepted] = 1;
      ++accepted;
      t += s->dt_min;
      m = std::min<int64_t>(2, m_max);
      bool stop = false;
      rc = run_output(s, accepted, t, 1, accepted == max_steps || t >= t_end * (1.0 - 1e-15), &stop);
      if (rc || stop) break;
      continue;
    }
    const int mi = static_cast<int>(m);
    // full step, not committed
    enqueue_trial(s, mi, s->stream);
    rc = sbiem_status(s, &st, nullptr, 1);
    if (rc) return rc;
    if (st) {
      m /= 2;
      continue;
    }
    CK(cudaMemcpyAsync(s->dfull, f.delta2, sizeof(double) * s->N, cudaMemcpyDeviceToDevice, s->stream));
    rc = snapshot(s, true);
    if (rc) return rc;
    ring_undo(s, mi, 0);
    enqueue_step(s, mi / 2, s->stream);
    enqueue_step(s, mi / 2, s->stream);
    launch_maxdiff(f.delta, s->dfull, s->N, s->d_err, s->stream);
    double eps = 0.0;
    CK(cudaMemcpyAsync(&eps, s->d_err, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    rc = sbiem_status(s, &st, nullptr, 1);
    if (rc) return rc;
    const double factor = eps > 0.0 ? 0.9 * std::cbrt(eps0 / eps) : HUGE_VAL;
    if (st || eps > eps0) {
      rc = snapshot(s, false);
      if (rc) return rc;
      ring_undo(s, mi, 1);
      int64_t mn = m / 2;
      if (!st)
        while (mn > 1 && static_cast<double>(mn) > factor * static_cast<double>(m)) mn /= 2;
      m = std::max<int64_t>(1, mn);
      continue;
    }
    if (m_hist) m_hist[accepted] = m;
    ++accepted;
    t += static_cast<double>(m) * s->dt_min;
    const int64_t m_acc = m;
    int64_t mn = m;
    while (static_cast<double>(mn * 2) <= factor * static_cast<double>(m) && mn < 2 * m) mn *= 2;
    while (mn > 1 && static_cast<double>(mn) > factor * static_cast<double>(m)) mn /= 2;
    m = std::max<int64_t>(1, std::min(mn, m_max));
    bool stop = false;
    rc = run_output(s, accepted, t, m_acc, accepted == max_steps || t >= t_end * (1.0 - 1e-15), &stop);
    if (rc || stop) break;
  }
  CK(cudaMemcpyAsync(&t, f.t, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (steps_out) *steps_out = accepted;
  if (m_next) *m_next = m;
  if (t_out) *t_out = t;
  return rc;
}

namespace {
// Page-locked (or NULL): host memory a captured copy may read or write.
bool host_pinned(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}
}  // namespace

int sbiem_step_host(sbiem_t s, double dt, const double* tau_load, double* V_out) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  int m;
  int rc = dt_to_m(s, dt, &m);
  if (rc) return rc;
  if (s->pslots == 0 && is_pow2(m) && m <= (1 << 30) && s->lag_m == m && host_pinned(tau_load) &&
      host_pinned(V_out)) {
    // steady overlapped stepping with pinned buffers: one graph launch and
    // one synchronization per step
    auto& hg = s->host_graph;
    if (!(hg.exec && hg.m == m && hg.tau == tau_load && hg.V == V_out)) {
      drop_host_graph(s);
      const size_t nb = sizeof(double) * s->N;
      CK(cudaStreamSynchronize(s->stream));
      CK(cudaStreamBeginCapture(s->own, cudaStreamCaptureModeThreadLocal));
      if (tau_load) cudaMemcpyAsync(s->f64.tau0, tau_load, nb, cudaMemcpyHostToDevice, s->own);
      if (s->fp32()) enqueue_step_lag_t<float>(s, s->f32, m, s->own);
      else enqueue_step_lag_t<double>(s, s->f64, m, s->own);
      if (V_out) cudaMemcpyAsync(V_out, s->f64.V, nb, cudaMemcpyDeviceToHost, s->own);
      cudaMemcpyAsync(s->h_status, s->f64.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->own);
      cudaError_t e1 = cudaGetLastError();
      cudaError_t e2 = cudaStreamEndCapture(s->own, &hg.def);
      if (e1 != cudaSuccess || e2 != cudaSuccess)
        return fail(SBIEM_ERR_CUDA,
                    std::string("graph capture: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
      CK(cudaGraphInstantiate(&hg.exec, hg.def, 0));
      hg.m = m;
      hg.tau = tau_load;
      hg.V = V_out;
    }
    CK(cudaGraphLaunch(hg.exec, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    const unsigned st = *s->h_status;
    if (st) {
      s->lag_m = -1;  // a rejected step left AT/AN of its start
      CK(cudaMemsetAsync(s->f64.status, 0, sizeof(unsigned), s->stream));
      return fail(status_to_code(st), "step rejected; state left at the start of the step");
    }
    return SBIEM_OK;
  }
  if (tau_load)
    CK(cudaMemcpyAsync(s->f64.tau0, tau_load, sizeof(double) * s->N, cudaMemcpyHostToDevice, s->stream));
  rc = sbiem_enqueue(s, dt, 1);
  if (rc) return rc;
  if (V_out) CK(cudaMemcpyAsync(V_out, s->f64.V, sizeof(double) * s->N, cudaMemcpyDeviceToHost, s->stream));
  uint32_t st;
  rc = sbiem_status(s, &st, nullptr, 1);
  if (rc) return rc;
  rc = status_to_code(st);
  if (rc) return fail(rc, "step rejected; state left at the start of the step");
  return SBIEM_OK;
}

int sbiem_get_state(sbiem_t s, double* delta, double* V, double* theta, double* tau_el,
                    double* sigma_el, double* t) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  const auto& f = s->f64;
  const size_t nb = sizeof(double) * s->N;
  if (delta) CK(cudaMemcpyAsync(delta, f.delta, nb, cudaMemcpyDeviceToHost, s->stream));
  if (V) CK(cudaMemcpyAsync(V, f.V, nb, cudaMemcpyDeviceToHost, s->stream));
  if (theta) CK(cudaMemcpyAsync(theta, f.th, nb, cudaMemcpyDeviceToHost, s->stream));
  std::vector<double> y;
  std::vector<float> y32;
  if (tau_el || sigma_el) {
    if (s->fp32()) {
      y32.resize(2 * s->N);
      CK(cudaMemcpyAsync(y32.data(), s->f32.y, sizeof(float) * 2 * s->N, cudaMemcpyDeviceToHost, s->stream));
    } else {
      y.resize(2 * s->N);
      CK(cudaMemcpyAsync(y.data(), f.y, sizeof(double) * 2 * s->N, cudaMemcpyDeviceToHost, s->stream));
    }
  }
  if (t) CK(cudaMemcpyAsync(t, f.t, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  for (int i = 0; i < s->N; ++i) {
    const double tr = s->fp32() ? static_cast<double>(y32.empty() ? 0.f : y32[2 * i]) : (y.empty() ? 0.0 : y[2 * i]);
    const double si = s->fp32() ? static_cast<double>(y32.empty() ? 0.f : y32[2 * i + 1]) : (y.empty() ? 0.0 : y[2 * i + 1]);
    if (tau_el) tau_el[i] = tr;
    if (sigma_el) sigma_el[i] = si;
  }
  return SBIEM_OK;
}

int sbiem_set_state(sbiem_t s, const double* delta, const double* V, const double* theta) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  s->lag_m = -1;
  auto& f = s->f64;
  const int N = s->N;
  const size_t nb = sizeof(double) * N;
  std::vector<double> Vh(N), th(N), Dc(N), psi(N), thd(N), xV(N), Vp(N);
  std::vector<uint8_t> pr(N);
  CK(cudaMemcpyAsync(Vh.data(), f.V, nb, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(th.data(), f.th, nb, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(Dc.data(), f.Dc, nb, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(Vp.data(), f.Vp, nb, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(pr.data(), f.presc, N, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (V) Vh.assign(V, V + N);
  for (int i = 0; i < N; ++i) {
    if (pr[i]) Vh[i] = Vp[i];  // prescribed elements keep their slip rate
    if (theta) th[i] = theta[i];
    if (!(th[i] > 0)) return fail(SBIEM_ERR_INVALID, "theta must be positive");
    psi[i] = std::log(th[i]);
    thd[i] = 1.0 - th[i] * Vh[i] / Dc[i];
    xV[i] = Vh[i] > 0.0 ? std::log(Vh[i]) : -745.0;
  }
  if (delta) CK(cudaMemcpyAsync(f.delta, delta, nb, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(f.V, Vh.data(), nb, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(f.psi, psi.data(), nb, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(f.th, th.data(), nb, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(f.thd, thd.data(), nb, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(f.xV, xV.data(), nb, cudaMemcpyHostToDevice, s->stream));
  int rc = recompute_spectral_sums(s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s->stream));
  return SBIEM_OK;
}

int sbiem_windows(sbiem_t s, int64_t* M) {
  if (!s || !M) return fail(SBIEM_ERR_INVALID, "NULL argument");
  std::memcpy(M, s->M.data(), sizeof(int64_t) * s->nmodes);
  return SBIEM_OK;
}

int sbiem_set_history(sbiem_t s, const double* hT, const double* hN) {
  if (!s || !hT || !hN) return fail(SBIEM_ERR_INVALID, "NULL argument");
  s->lag_m = -1;
  const int64_t tot = s->total_slots;
  if (tot == 0) return SBIEM_OK;
  std::vector<int32_t> heads(s->nmodes, 0);
  if (s->fp32()) {
    std::vector<float4> buf(tot);
    for (int64_t i = 0; i < tot; ++i)
      buf[i] = make_float4(static_cast<float>(hT[2 * i]), static_cast<float>(hT[2 * i + 1]),
                           static_cast<float>(hN[2 * i]), static_cast<float>(hN[2 * i + 1]));
    CK(cudaMemcpyAsync(s->f32.ring, buf.data(), sizeof(float4) * tot, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->f32.head, heads.data(), sizeof(int32_t) * s->nmodes, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  } else {
    std::vector<Slot64> buf(tot);
    for (int64_t i = 0; i < tot; ++i) {
      buf[i].t = make_double2(hT[2 * i], hT[2 * i + 1]);
      buf[i].n = make_double2(hN[2 * i], hN[2 * i + 1]);
    }
    CK(cudaMemcpyAsync(s->f64.ring, buf.data(), sizeof(Slot64) * tot, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->f64.head, heads.data(), sizeof(int32_t) * s->nmodes, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  return SBIEM_OK;
}

int sbiem_set_history_device(sbiem_t s, const void* hT, const void* hN, int32_t values_fp32) {
  if (!s || (values_fp32 != 0 && values_fp32 != 1)) return fail(SBIEM_ERR_INVALID, "NULL handle or bad flag");
  s->lag_m = -1;
  const int64_t tot = s->total_slots;
  if (tot == 0) return SBIEM_OK;  // no history (quasi-dynamic limit): nothing to read
  if (!hT || !hN) return fail(SBIEM_ERR_INVALID, "NULL history array");
  std::vector<int32_t> heads(s->nmodes, 0);
  if (s->fp32()) {
    launch_set_ring<float>(s->f32.ring, hT, hN, values_fp32 == 1, tot, s->sm_count, s->stream);
    CK(cudaMemcpyAsync(s->f32.head, heads.data(), sizeof(int32_t) * s->nmodes, cudaMemcpyHostToDevice, s->stream));
  } else {
    launch_set_ring<double>(s->f64.ring, hT, hN, values_fp32 == 1, tot, s->sm_count, s->stream);
    CK(cudaMemcpyAsync(s->f64.head, heads.data(), sizeof(int32_t) * s->nmodes, cudaMemcpyHostToDevice, s->stream));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s->stream));
  return SBIEM_OK;
}

int sbiem_get_history(sbiem_t s, double* hT, double* hN) {
  if (!s || !hT || !hN) return fail(SBIEM_ERR_INVALID, "NULL argument");
  const int64_t tot = s->total_slots;
  if (tot == 0) return SBIEM_OK;
  std::vector<int32_t> heads(s->nmodes);
  CK(cudaMemcpyAsync(heads.data(), s->f64.head, sizeof(int32_t) * s->nmodes, cudaMemcpyDeviceToHost, s->stream));
  std::vector<Slot64> b64;
  std::vector<float4> b32;
  if (s->fp32()) {
    b32.resize(tot);
    CK(cudaMemcpyAsync(b32.data(), s->f32.ring, sizeof(float4) * tot, cudaMemcpyDeviceToHost, s->stream));
  } else {
    b64.resize(tot);
    CK(cudaMemcpyAsync(b64.data(), s->f64.ring, sizeof(Slot64) * tot, cudaMemcpyDeviceToHost, s->stream));
  }
  CK(cudaStreamSynchronize(s->stream));
  for (int n = 0; n < s->nmodes; ++n) {
    const int64_t Rn = s->Rn[n], off = s->ring_off[n];
    for (int64_t i = 0; i < Rn; ++i) {
      const int64_t src = off + (heads[n] + i) % Rn, dst = off + i;
      if (s->fp32()) {
        hT[2 * dst] = b32[src].x;
        hT[2 * dst + 1] = b32[src].y;
        hN[2 * dst] = b32[src].z;
        hN[2 * dst + 1] = b32[src].w;
      } else {
        hT[2 * dst] = b64[src].t.x;
        hT[2 * dst + 1] = b64[src].t.y;
        hN[2 * dst] = b64[src].n.x;
        hN[2 * dst + 1] = b64[src].n.y;
      }
    }
  }
  return SBIEM_OK;
}

int sbiem_history_sums(sbiem_t s, int64_t m, double* AT, double* AN) {
  if (!s || !AT || !AN || m < 1 || m > (int64_t(1) << 30)) return fail(SBIEM_ERR_INVALID, "bad argument");
  const int mi = static_cast<int>(m);
  if (s->fp32()) launch_history<float>(s->f32, mi, s->hist_grid, s->stream);
  else launch_history<double>(s->f64, mi, s->hist_grid, s->stream);
  CK(cudaGetLastError());
  s->lag_m = mi;  // AT/AN now hold the sums of a step of m from this state
  const size_t nb = sizeof(double2) * s->nmodes;
  CK(cudaMemcpyAsync(AT, s->f64.AT, nb, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(AN, s->f64.AN, nb, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return SBIEM_OK;
}

int sbiem_history_enqueue_marked(sbiem_t s, int64_t m, void* sweep_done) {
  if (!s || m < 1 || m > (int64_t(1) << 30)) return fail(SBIEM_ERR_INVALID, "bad argument");
  const int mi = static_cast<int>(m);
  cudaEvent_t ev = static_cast<cudaEvent_t>(sweep_done);
  if (s->fp32()) launch_history<float>(s->f32, mi, s->hist_grid, s->stream, ev);
  else launch_history<double>(s->f64, mi, s->hist_grid, s->stream, ev);
  CK(cudaGetLastError());
  s->lag_m = mi;
  return SBIEM_OK;
}

int sbiem_history_enqueue(sbiem_t s, int64_t m) { return sbiem_history_enqueue_marked(s, m, nullptr); }

int sbiem_read_probe(const void* data, int64_t bytes, float* sink, void* stream) {
  if (!data || !sink || bytes <= 0 || (bytes & 15) || (reinterpret_cast<uintptr_t>(data) & 15))
    return fail(SBIEM_ERR_INVALID, "read probe: null or misaligned pointer or size");
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  launch_read_probe(data, bytes, sink, sms, static_cast<cudaStream_t>(stream));
  CK(cudaGetLastError());
  return SBIEM_OK;
}

namespace {
void drop_graphs(sbiem_s* s) {
  cudaStreamSynchronize(s->stream);
  drop_host_graph(s);
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : s->graph_defs) cudaGraphDestroy(kv.second);
  for (auto& kv : s->lag_graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : s->lag_defs) cudaGraphDestroy(kv.second);
  s->graphs.clear();
  s->graph_defs.clear();
  s->lag_graphs.clear();
  s->lag_defs.clear();
  s->pnodes.clear();
}
}  // namespace

int sbiem_set_mlp(sbiem_t s, const float* params) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  drop_graphs(s);
  if (!params) {
    s->f64.mlp = nullptr;
    s->f32.mlp = nullptr;
    return SBIEM_OK;
  }
  if (!s->mlp) {
    s->mlp = static_cast<MlpDev*>(dev_alloc(s, sizeof(MlpDev)));
    if (!s->mlp) return fail(SBIEM_ERR_NOMEM, "network allocation failed");
  }
  int rc = mlp_deploy(params, s->mlp, s->stream);
  if (rc) return fail(rc, "network upload failed");
  s->f64.mlp = s->mlp;
  s->f32.mlp = s->mlp;
  return SBIEM_OK;
}

int sbiem_harvest_enable(sbiem_t s, int64_t capacity) {
  if (!s || capacity < 0) return fail(SBIEM_ERR_INVALID, "bad argument");
  drop_graphs(s);
  if (capacity == 0) {
    s->f64.harvest = s->f32.harvest = nullptr;
    return SBIEM_OK;
  }
  if (capacity > s->harvest_cap) {
    s->harvest = static_cast<float*>(dev_alloc(s, sizeof(float) * 6 * static_cast<size_t>(capacity)));
    if (!s->harvest_count)
      s->harvest_count = static_cast<unsigned long long*>(dev_alloc(s, sizeof(unsigned long long)));
    if (!s->harvest || !s->harvest_count) return fail(SBIEM_ERR_NOMEM, "harvest buffer allocation failed");
    s->harvest_cap = capacity;
  }
  CK(cudaMemsetAsync(s->harvest_count, 0, sizeof(unsigned long long), s->stream));
  for (auto* f : {&s->f64}) {
    f->harvest = s->harvest;
    f->harvest_count = s->harvest_count;
    f->harvest_cap = s->harvest_cap;
  }
  s->f32.harvest = s->harvest;
  s->f32.harvest_count = s->harvest_count;
  s->f32.harvest_cap = s->harvest_cap;
  return SBIEM_OK;
}

int sbiem_harvest_read(sbiem_t s, float* rows_out, int64_t max_rows, int64_t* rows, int reset) {
  if (!s || max_rows < 0) return fail(SBIEM_ERR_INVALID, "bad argument");
  unsigned long long cnt = 0;
  if (s->harvest_count) {
    CK(cudaMemcpyAsync(&cnt, s->harvest_count, sizeof(cnt), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  int64_t n = std::min<int64_t>(static_cast<int64_t>(std::min<unsigned long long>(cnt, s->harvest_cap)), max_rows);
  if (rows_out && n > 0)
    CK(cudaMemcpy(rows_out, s->harvest, sizeof(float) * 6 * n, cudaMemcpyDeviceToHost));
  if (rows) *rows = static_cast<int64_t>(std::min<unsigned long long>(cnt, s->harvest_cap));
  if (reset && s->harvest_count) CK(cudaMemsetAsync(s->harvest_count, 0, sizeof(unsigned long long), s->stream));
  return SBIEM_OK;
}

int sbiem_probe_enable(sbiem_t s, int nslots) {
  if (!s || nslots < 0 || nslots > (1 << 20)) return fail(SBIEM_ERR_INVALID, "bad argument");
  CK(cudaStreamSynchronize(s->stream));
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : s->graph_defs) cudaGraphDestroy(kv.second);
  s->graphs.clear();
  s->graph_defs.clear();
  s->pnodes.clear();
  for (auto& e : s->pev)
    if (e) cudaEventDestroy(e);
  s->pev.assign(static_cast<size_t>(4) * nslots, nullptr);
  for (auto& e : s->pev) CK(cudaEventCreate(&e));
  s->pslots = nslots;
  s->pcount = 0;
  s->pcur = 0;
  return SBIEM_OK;
}

int sbiem_probe_read(sbiem_t s, int slot, float* ms_step, float* ms_history) {
  if (!s || !s->pslots || slot < 0 || slot >= s->pslots) return fail(SBIEM_ERR_INVALID, "probe not enabled or bad slot");
  cudaEvent_t* e = &s->pev[4 * slot];
  CK(cudaEventSynchronize(e[3]));
  float a = 0.f, b = 0.f;
  CK(cudaEventElapsedTime(&a, e[0], e[3]));
  CK(cudaEventElapsedTime(&b, e[1], e[2]));
  if (ms_step) *ms_step = a;
  if (ms_history) *ms_history = b;
  return SBIEM_OK;
}

int sbiem_newton_totals(sbiem_t s, int64_t* iters, int64_t* solves, int reset) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  unsigned long long v[2] = {0ull, 0ull};
  CK(cudaMemcpyAsync(v, s->f64.it_total, sizeof(v), cudaMemcpyDeviceToHost, s->stream));
  if (reset) CK(cudaMemsetAsync(s->f64.it_total, 0, sizeof(v), s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (iters) *iters = static_cast<int64_t>(v[0]);
  if (solves) *solves = static_cast<int64_t>(v[1]);
  return SBIEM_OK;
}

int sbiem_newton_stats(sbiem_t s, int64_t* iters_sum, int32_t* iters_max) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  unsigned long long sum = 0;
  int mx = 0;
  CK(cudaMemcpyAsync(&sum, s->f64.it_sum, sizeof(sum), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(&mx, s->f64.it_max, sizeof(mx), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (iters_sum) *iters_sum = static_cast<int64_t>(sum);
  if (iters_max) *iters_max = mx;
  return SBIEM_OK;
}

int sbiem_footprint(sbiem_t s, int64_t* hist_bytes, int64_t* device_bytes) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  const int64_t slot = s->fp32() ? 16 : 32, wb = s->fp32() ? 8 : 16;
  // weights stream only for the modes that do not evaluate them on chip
  int64_t streamed = 0;
  for (int n = 1; n < s->nmodes; ++n) {
    const double ds = s->p.cs * (2.0 * M_PI * n / s->L) * s->dt_min;
    if (!(s->fp32() && s->f32.gen_ds_max > 0.0f && static_cast<float>(ds) <= s->f32.gen_ds_max))
      streamed += s->Rn[n];
  }
  if (hist_bytes) *hist_bytes = s->total_slots * slot + streamed * wb;
  if (device_bytes) *device_bytes = s->device_bytes;
  return SBIEM_OK;
}

int sbiem_set_wait_limit(sbiem_t s, int64_t polls) {
  if (!s || polls < 0) return fail(SBIEM_ERR_INVALID, "NULL handle or negative limit");
  CK(cudaStreamSynchronize(s->stream));
  s->spin_limit = polls;
  s->f64.spin_limit = polls;
  s->f32.spin_limit = polls;
  drop_graphs(s);
  s->lag_m = -1;
  return SBIEM_OK;
}

int sbiem_get_sweep(sbiem_t s, int32_t* shape, double* gen_ds_max, int32_t* ctas_per_sm, int32_t* lag_ctas_per_sm,
                    double* table_err) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  if (shape) *shape = s->sweep_shape;
  if (gen_ds_max) *gen_ds_max = s->fp32() ? s->f32.gen_ds_max : 0.0;
  if (ctas_per_sm) *ctas_per_sm = s->hist_grid / (s->sm_count > 0 ? s->sm_count : 1);
  if (lag_ctas_per_sm) *lag_ctas_per_sm = s->lag_grid / (s->sm_count > 0 ? s->sm_count : 1);
  if (table_err) *table_err = s->gen_pieces > 0 ? s->gen_err : -1.0;
  return SBIEM_OK;
}

int sbiem_set_sweep(sbiem_t s, int32_t shape, double gen_ds_max, int32_t ctas_per_sm) {
  if (!s) return fail(SBIEM_ERR_INVALID, "NULL handle");
  if (shape < 0 || shape > 4 || sweep_chunk_slots(s->p.precision, shape) != s->chunk_slots)
    return fail(SBIEM_ERR_INVALID, "shape must keep the handle's chunk length (" + std::to_string(s->chunk_slots) +
                                       " lags)");
  if (!(gen_ds_max >= 0.0)) return fail(SBIEM_ERR_INVALID, "gen_ds_max must be >= 0");
  if (gen_ds_max > 0.0 && s->gen_pieces == 0)
    return fail(SBIEM_ERR_UNSUPPORTED, "no on-chip weight table (FP64 form, exact quadrature, or windows past it)");
  if (ctas_per_sm < 0) return fail(SBIEM_ERR_INVALID, "ctas_per_sm must be >= 0");
  CK(cudaStreamSynchronize(s->stream));
  s->sweep_shape = shape;
  s->gen_ds_max = static_cast<float>(std::min(gen_ds_max, kGenDsBlock4Max));
  s->sweep_ctas = ctas_per_sm;
  s->lag_ctas = 0;  // the overlapped sweep's grid follows the rule again (sbiem_tune times it)
  sweep_config(s);
  drop_graphs(s);
  s->lag_m = -1;
  return SBIEM_OK;
}

int sbiem_set_lag_sweep(sbiem_t s, int32_t lag_ctas_per_sm) {
  if (!s || lag_ctas_per_sm < 0) return fail(SBIEM_ERR_INVALID, "NULL handle or negative CTA count");
  CK(cudaStreamSynchronize(s->stream));
  s->lag_ctas = lag_ctas_per_sm;
  sweep_config(s);
  drop_graphs(s);
  s->lag_m = -1;
  return SBIEM_OK;
}

int sbiem_tune(sbiem_t s, int reps, int32_t* shape_out, double* gen_out, int32_t* ctas_out, float* ms_out) {
  if (!s || reps < 1) return fail(SBIEM_ERR_INVALID, "bad argument");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // thresholds of the on-chip weights: none, then 1/8 .. 1 of the largest
  // s step the on-chip blocks allow
  std::vector<float> thr = {0.0f};
  if (s->gen_pieces > 0)
    for (double v : {kGenDsBlockMax / 8.0, kGenDsBlockMax / 4.0, kGenDsBlockMax / 2.0, kGenDsBlockMax,
                     kGenDsBlock4Max})
      thr.push_back(static_cast<float>(v));
  float best = 1e30f;
  int bshape = s->sweep_shape, bctas = 0;
  float bthr = s->gen_ds_max;
  struct ShapeBest {
    float ms, thr;
    int ctas;
  };
  ShapeBest shape_best[5];
  for (auto& x : shape_best) x = {1e30f, 0.0f, 0};
  for (int shape = 0; shape <= 4; ++shape) {
    if (sweep_chunk_slots(s->p.precision, shape) != s->chunk_slots) continue;
    for (float t : thr) {
      const int lim = s->fp32() ? sweep_blocks_per_sm<float>(shape, t > 0.0f)
                                : sweep_blocks_per_sm<double>(shape, false);
      for (int c = 1; c <= lim; ++c) {
        s->sweep_shape = shape;
        s->gen_ds_max = t;
        s->sweep_ctas = c;
        sweep_config(s);
        std::vector<float> tm;
        for (int k = 0; k <= reps; ++k) {
          CK(cudaEventRecord(e0, s->stream));
          if (s->fp32()) launch_history<float>(s->f32, 1, s->hist_grid, s->stream);
          else launch_history<double>(s->f64, 1, s->hist_grid, s->stream);
          CK(cudaEventRecord(e1, s->stream));
          CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          if (k > 0) tm.push_back(ms);  // the first launch is untimed
        }
        std::sort(tm.begin(), tm.end());
        const float med = tm[tm.size() / 2];
        if (med < best) {
          best = med;
          bshape = shape;
          bthr = t;
          bctas = c;
        }
        if (med < shape_best[shape].ms) shape_best[shape] = {med, t, c};
      }
    }
  }
  // With the four-kernel passes (FP32, N > kFusedMaxN) the sweep that is
  // fastest alone need not give the fastest step: at N = 65536 and 262144
  // two two-stage CTAs per SM (shape 3) leave the passes room beside the
  // next step's sweep (steps 0.271 and 1.113 ms, against 0.292 and 1.150 ms
  // for four one-stage CTAs, the faster sweep alone).  So the best setting
  // of each shape is timed over real overlapped steps, each undone after
  // its timing (state snapshot and the overwritten ring slot restored), and
  // the fastest step is kept.
  if (s->fp32() && s->N > kFusedMaxN && s->nmodes > 0) {
    bool ok = ensure_snapshot(s);
    if (ok && !s->tune_slots) {
      s->tune_slots = dev_alloc(s, sizeof(Slot32) * static_cast<size_t>(s->nmodes));
      ok = s->tune_slots != nullptr;
    }
    if (!ok) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return nomem(s, "autotuner snapshot");
    }
    unsigned st0 = 0;
    unsigned long long tot0[2] = {0ull, 0ull};
    CK(cudaMemcpyAsync(&st0, s->f64.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(tot0, s->f64.it_total, sizeof(tot0), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    float step_best = 1e30f;
    int sb_shape = bshape, sb_ctas = bctas;
    float sb_thr = bthr;
    for (int shape = 0; shape <= 4; ++shape) {
      if (shape_best[shape].ms >= 1e29f) continue;
      int rc0 = sbiem_set_sweep(s, shape, shape_best[shape].thr, shape_best[shape].ctas);
      if (rc0 == SBIEM_OK) rc0 = lag_graph(s, 1);
      if (rc0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc0;
      }
      std::vector<float> tm;
      for (int k = 0; k <= reps; ++k) {
        int rcs = snapshot(s, true);
        if (rcs) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return rcs;
        }
        launch_slot_swap<float>(s->f32, s->tune_slots, 0, s->stream);
        launch_history<float>(s->f32, 1, s->hist_grid, s->stream);  // this step's sums (the prologue)
        CK(cudaEventRecord(e0, s->stream));
        CK(cudaGraphLaunch(s->lag_graphs[1], s->stream));
        CK(cudaEventRecord(e1, s->stream));
        CK(cudaEventSynchronize(e1));
        rcs = snapshot(s, false);
        if (rcs) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return rcs;
        }
        launch_slot_swap<float>(s->f32, s->tune_slots, 1, s->stream);
        CK(cudaMemcpyAsync(s->f64.status, &st0, sizeof(unsigned), cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (k > 0) tm.push_back(ms);
      }
      std::sort(tm.begin(), tm.end());
      if (tm[tm.size() / 2] < step_best) {
        step_best = tm[tm.size() / 2];
        sb_shape = shape;
        sb_thr = shape_best[shape].thr;
        sb_ctas = shape_best[shape].ctas;
      }
    }
    CK(cudaMemcpy(s->f64.it_total, tot0, sizeof(tot0), cudaMemcpyHostToDevice));
    bshape = sb_shape;
    bthr = sb_thr;
    bctas = sb_ctas;
    best = shape_best[bshape].ms;
  }
  int rc = sbiem_set_sweep(s, bshape, bthr, bctas);
  if (rc) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
  }
  // the overlapped step: the next step's sweep (into BT/BN) on the side
  // stream beside this step's two passes (their results stay staged), timed
  // together for 1 .. (occupancy limit) sweep CTAs per SM; nothing is
  // committed, and the status word the passes may set is put back.  Only
  // where the passes are one-launch kernels that fit beside the sweep (FP32,
  // N <= kFusedMaxN): with the four-kernel passes the full grid is best (per
  // step, 3 against 4 CTAs per SM: 1.34 against 1.15 ms at N = 262144, 0.31
  // against 0.27-0.29 ms at N = 65536), and this proxy, which leaves out the
  // commit and the graph, picked 3 at N = 65536.
  if (s->fp32() && s->N <= kFusedMaxN) {
    unsigned st0 = 0;
    CK(cudaMemcpyAsync(&st0, s->f64.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->lag_ctas = 0;
    sweep_config(s);
    const int lim = s->fp32() ? sweep_blocks_per_sm<float>(s->lag_shape, s->f32.gen_ds_max > 0.0f)
                              : sweep_blocks_per_sm<double>(s->lag_shape, false);
    float lbest = 1e30f;
    int lb = 0;
    // nine timed launches at least: the candidates' totals are close (with
    // five, the N = 65536 rough cycle's step came out at 0.27 or 0.31 ms
    // from run to run)
    const int reps_lag = std::max(reps, 9);
    for (int c = 1; c <= lim; ++c) {
      s->lag_ctas = c;
      sweep_config(s);
      std::vector<float> tm;
      for (int k = 0; k <= reps_lag; ++k) {
        CK(cudaEventRecord(e0, s->stream));
        // in the order of the step graph (the sweep after the pass-1
        // spectral kernel has started)
        auto both = [&](const auto& f) {
          using R = typename std::decay_t<decltype(f)>::Real;
          cudaEventRecord(s->ev_fork, s->stream);
          launch_spectral<R>(f, 1, 1, s->stream, s->ev_started);
          cudaStreamWaitEvent(s->side, s->ev_fork, 0);
          cudaStreamWaitEvent(s->side, s->ev_started, 0);
          launch_history_ahead<R>(f, 1, s->lag_grid, s->side);
          launch_newton<R>(f, 1, 1, s->stream);
          launch_pass<R>(f, 2, 1, s->stream);
        };
        if (s->fp32()) both(s->f32);
        else both(s->f64);
        CK(cudaGetLastError());
        CK(cudaEventRecord(s->ev_join, s->side));
        CK(cudaStreamWaitEvent(s->stream, s->ev_join, 0));
        CK(cudaEventRecord(e1, s->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (k > 0) tm.push_back(ms);
      }
      std::sort(tm.begin(), tm.end());
      if (tm[tm.size() / 2] < lbest) {
        lbest = tm[tm.size() / 2];
        lb = c;
      }
    }
    CK(cudaMemcpyAsync(s->f64.status, &st0, sizeof(unsigned), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->lag_ctas = lb;
    sweep_config(s);
    drop_graphs(s);
    s->lag_m = -1;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (shape_out) *shape_out = bshape;
  if (gen_out) *gen_out = bthr;
  if (ctas_out) *ctas_out = bctas;
  if (ms_out) *ms_out = best;
  return SBIEM_OK;
}

}  // extern "C"

// ============================================================ ensembles
// A batch steps many faults at once: one history-convolution launch over the
// chunks of every member, then per group of equal N one launch of each pass
// kernel with one member per blockIdx.y, the groups as parallel graph branches.
struct sbiem_batch_s {
  std::vector<sbiem_s*> members;  // grouped order
  std::vector<int> order;         // grouped position -> caller index
  bool fp32 = false;
  int sm_count = 0, hist_grid = 0, per_sm = 1;
  int64_t chunk_slots = 0;
  cudaStream_t stream = nullptr, own = nullptr;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> fork_join;
  cudaStream_t side = nullptr;                       // overlapped history sweep
  cudaEvent_t ev_fork = nullptr, ev_side = nullptr;
  int lag_grid = 0;
  bool overlap = false;  // sweep the next step beside the passes (sbiem_batch_tune / set_overlap)
  struct Group {
    int N, first, count;
    FftGeom g;
  };
  std::vector<Group> groups;
  void* fs = nullptr;  // DevFault<R>[members] on the device
  Chunk* chunks = nullptr;      // members' chunk tables, concatenated (member in Chunk::pad)
  int nchunks = 0;
  double4* partial = nullptr;   // sweep partials per chunk
  int2* fc = nullptr;           // (first chunk, chunks) of each (member, mode) pair, mm order
  // chunk tables by chunk length (the autotuner tries every shape's); the
  // pointers above are those of the length in force (chunk_slots)
  struct ChunkSet {
    Chunk* chunks;
    double4* partial;
    int2* fc;
    int n;
  };
  std::map<int64_t, ChunkSet> sets;
  int2* mm = nullptr;           // (member, mode) pairs of the per-mode sums
  int TM = 0;
  int shape = 0;                // sweep shape shared by the members
  // on-chip weights (FP32): one table serves every member when they share
  // c_s/c_p and dt_min (the weights are then one function of s)
  const float4* wtab = nullptr;
  int gen_pieces = 0;
  bool gen = false;
  float gen_ds_max = 0.0f;  // in force while gen
  int per_sm_plain = 1, per_sm_gen = 1;
  // the history convolution as one persistent cooperative launch: its grid
  // barrier's counter and epoch (device), and the barrier's poll limit
  unsigned* bar = nullptr;
  long long bar_limit = SBIEM_WAIT_LIMIT_DEFAULT;
  // members whose weights are equal read one copy of them (the first such
  // member's); with any shared the sweep copies ring slots evict-first
  int distinct_weights = 0;
  bool shared_weights = false;
  bool persistent = true;  // one cooperative launch; false: sweep launch + sum launch
  std::vector<void*> allocs;
  cudaGraphExec_t graph = nullptr;
  cudaGraph_t graph_def = nullptr;
};

namespace {

void batch_free(sbiem_batch_s* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->graph_def) cudaGraphDestroy(b->graph_def);
  b->graph = nullptr;
  b->graph_def = nullptr;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
  for (auto e : b->fork_join) cudaEventDestroy(e);
  for (auto st : b->branch) cudaStreamDestroy(st);
  if (b->side) {
    cudaStreamSynchronize(b->side);
    cudaStreamDestroy(b->side);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_side) cudaEventDestroy(b->ev_side);
  if (b->own) cudaStreamDestroy(b->own);
}

void* batch_alloc(sbiem_batch_s* b, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
  b->allocs.push_back(p);
  return p;
}

// Members with equal N, length, c_s, c_p, dt_min, windows (both fields),
// quadrature and precision have bitwise equal weights: the weight builder
// reads nothing else.
bool same_weights(const sbiem_s* a, const sbiem_s* b) {
  return a->fp32() == b->fp32() && a->p.N == b->p.N && a->L == b->L && a->dt_min == b->dt_min &&
         a->p.cs == b->p.cs && a->p.cp == b->p.cp && a->p.quadrature == b->p.quadrature && a->MT == b->MT &&
         a->MN == b->MN;
}

// Members whose wavenumbers coincide share weights across sizes too: with
// equal dx, c_s, c_p, dt_min, quadrature and precision, mode n of N and mode
// n N'/N of N' = 2^p N have the same k (k = 2 pi n / L bitwise: scaling n
// and L by 2^p is exact), so the same weights dt C(c_s k (j + 1/2) dt) as
// far as both windows reach.  With one cutting plane (each field's window
// the mode's) a member whose every window is no longer than the larger
// member's reads a prefix of that member's weight run.  Returns N'/N when
// member r can read member c's weights, else 0.
int64_t weight_ratio(const sbiem_s* r, const sbiem_s* c) {
  if (r->fp32() != c->fp32() || r->p.cs != c->p.cs || r->p.cp != c->p.cp || r->dt_min != c->dt_min ||
      r->p.quadrature != c->p.quadrature)
    return 0;
  if (c->p.N < r->p.N || c->p.N % r->p.N != 0) return 0;
  const int64_t ratio = c->p.N / r->p.N;
  if ((ratio & (ratio - 1)) != 0 || r->L * static_cast<double>(ratio) != c->L) return 0;
  if (r->MT != r->MN || c->MT != c->MN) return 0;
  for (int n = 1; n < r->nmodes; ++n)
    if (r->M[n] > c->M[static_cast<size_t>(n) * ratio]) return 0;
  return ratio;
}

// Ensemble chunk table: the members' own chunk tables one after another
// (member index in Chunk::pad), each member's first chunk, the (member,
// mode) list of the per-mode sums; member descriptors on the device.
// The ensemble's chunk table for chunks of at most `slots` lags (built once
// per length, then reused): every member's modes in order, each mode's ring
// cut into runs of `slots` lags (member in Chunk::pad), and per (member,
// mode) pair its first chunk and count.  Makes that length the one in force.
int batch_use_chunks(sbiem_batch_s* b, int64_t slots) {
  auto it = b->sets.find(slots);
  if (it == b->sets.end()) {
    std::vector<Chunk> ch;
    std::vector<int2> fc;
    for (size_t r = 0; r < b->members.size(); ++r) {
      const sbiem_s* s = b->members[r];
      for (int n = 0; n < s->nmodes; ++n) {
        const int64_t cnt = (s->Rn[n] + slots - 1) / slots;
        fc.push_back(make_int2(static_cast<int>(ch.size()), static_cast<int>(cnt)));
        for (int64_t c = 0; c < cnt; ++c) {
          Chunk x{};
          x.mode = n;
          x.first = static_cast<int32_t>(ch.size() - c);
          x.count = static_cast<int32_t>(cnt);
          x.pad = static_cast<int32_t>(r);
          x.i0 = c * slots;
          x.i1 = std::min<int64_t>((c + 1) * slots, s->Rn[n]);
          ch.push_back(x);
        }
      }
      if (ch.size() > static_cast<size_t>(1) << 30) return fail(SBIEM_ERR_INVALID, "batch: too many chunks");
    }
    sbiem_batch_s::ChunkSet cs{};
    cs.n = static_cast<int>(ch.size());
    cs.chunks = static_cast<Chunk*>(batch_alloc(b, sizeof(Chunk) * std::max<size_t>(ch.size(), 1)));
    cs.partial = static_cast<double4*>(batch_alloc(b, sizeof(double4) * std::max<size_t>(ch.size(), 1)));
    cs.fc = static_cast<int2*>(batch_alloc(b, sizeof(int2) * std::max<size_t>(fc.size(), 1)));
    if (!cs.chunks || !cs.partial || !cs.fc) return fail(SBIEM_ERR_NOMEM, "batch: device allocation failed (chunks)");
    if (!ch.empty()) CK(cudaMemcpy(cs.chunks, ch.data(), sizeof(Chunk) * ch.size(), cudaMemcpyHostToDevice));
    if (!fc.empty()) CK(cudaMemcpy(cs.fc, fc.data(), sizeof(int2) * fc.size(), cudaMemcpyHostToDevice));
    it = b->sets.emplace(slots, cs).first;
  }
  b->chunks = it->second.chunks;
  b->partial = it->second.partial;
  b->fc = it->second.fc;
  b->nchunks = it->second.n;
  b->chunk_slots = slots;
  return SBIEM_OK;
}

template <class R>
int batch_build(sbiem_batch_s* b) {
  std::vector<int2> mm;
  for (size_t r = 0; r < b->members.size(); ++r)
    for (int n = 0; n < b->members[r]->nmodes; ++n) mm.push_back(make_int2(static_cast<int>(r), n));
  b->mm = static_cast<int2*>(batch_alloc(b, sizeof(int2) * std::max<size_t>(mm.size(), 1)));
  b->fs = batch_alloc(b, sizeof(DevFault<R>) * b->members.size());
  b->bar = static_cast<unsigned*>(batch_alloc(b, 2 * sizeof(unsigned)));
  if (!b->mm || !b->fs || !b->bar) return fail(SBIEM_ERR_NOMEM, "batch: device allocation failed");
  CK(cudaStreamSynchronize(b->stream));
  const int rc_ch = batch_use_chunks(b, b->chunk_slots);
  if (rc_ch) return rc_ch;
  CK(cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned), b->stream));
  std::vector<DevFault<R>> fs(b->members.size());
  for (size_t r = 0; r < b->members.size(); ++r) {
    DevFault<R> f;
    if constexpr (sizeof(R) == 8) f = b->members[r]->f64;
    else f = b->members[r]->f32;
    f.newton_epw = 32;  // the batched Newton launch covers 32 elements per warp
    fs[r] = f;
  }
  // weights: each member reads those of the largest member it can (itself
  // when none); members of one size share one offset table into it
  {
    const size_t nm = b->members.size();
    std::map<std::pair<size_t, int64_t>, int64_t*> maps;  // (source member, N) -> device offsets
    for (size_t r = 0; r < nm; ++r) {
      const sbiem_s* sr = b->members[r];
      size_t src = r;
      int64_t ratio = 1;
      for (size_t q = 0; q < nm; ++q) {
        const int64_t t = weight_ratio(sr, b->members[q]);
        if (t > ratio || (t == ratio && t > 0 && q < src && b->members[q]->p.N == b->members[src]->p.N)) {
          src = q;
          ratio = t;
        }
      }
      if (src == r) continue;
      if (ratio == 1 && same_weights(sr, b->members[src])) {
        fs[r].w = fs[src].w;
        fs[r].w_off = fs[src].w_off;
        fs[r].wgen = fs[src].wgen;
        continue;
      }
      auto key = std::make_pair(src, static_cast<int64_t>(sr->p.N));
      auto it = maps.find(key);
      if (it == maps.end()) {
        const sbiem_s* sc = b->members[src];
        std::vector<int64_t> wo(static_cast<size_t>(sr->nmodes) + 1);
        for (int n = 0; n <= sr->nmodes; ++n)
          wo[n] = sc->w_off[std::min<size_t>(static_cast<size_t>(n) * ratio, static_cast<size_t>(sc->nmodes))];
        int64_t* d = static_cast<int64_t*>(batch_alloc(b, sizeof(int64_t) * wo.size()));
        if (!d) return fail(SBIEM_ERR_NOMEM, "batch: device allocation failed (weight offsets)");
        CK(cudaMemcpy(d, wo.data(), sizeof(int64_t) * wo.size(), cudaMemcpyHostToDevice));
        it = maps.emplace(key, d).first;
      }
      fs[r].w = fs[src].w;
      fs[r].w_off = it->second;
    }
  }
  b->distinct_weights = 0;
  for (size_t r = 0; r < fs.size(); ++r) {
    bool first = true;
    for (size_t q = 0; q < r && first; ++q) first = fs[q].w != fs[r].w;
    b->distinct_weights += first ? 1 : 0;
  }
  b->shared_weights = b->distinct_weights < static_cast<int>(fs.size());
  CK(cudaMemcpyAsync(b->mm, mm.data(), sizeof(int2) * mm.size(), cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->fs, fs.data(), sizeof(DevFault<R>) * fs.size(), cudaMemcpyHostToDevice, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  b->TM = static_cast<int>(mm.size());
  return SBIEM_OK;
}

// Whole-window sums of every member (AT, AN), or with ahead = true the next
// step's sums without its newest interval (BT, BN; weights shifted by 2).
template <class R>
void batch_history(sbiem_batch_s* b, cudaStream_t st, bool ahead = false) {
  // one persistent launch: every CTA resident (the grid never exceeds the
  // occupancy the CTAs per SM were chosen within) and at least one chunk each
  int grid = ahead ? b->lag_grid : b->hist_grid;
  const bool gen = sizeof(R) == 4 && b->gen;
  const int resident = b->sm_count * std::max(1, persist_blocks_per_sm<R>(b->shape, gen));
  if (grid > resident) grid = resident;
  if (grid > b->nchunks) grid = b->nchunks > 0 ? b->nchunks : 1;
  if (!b->persistent) {
    launch_history_batch<R>(static_cast<const DevFault<R>*>(b->fs), b->chunks, b->nchunks, b->partial, b->mm,
                            b->TM, b->fc, b->shape, grid, ahead ? 2 : 1, st, ahead, b->gen ? b->wtab : nullptr,
                            b->gen ? b->gen_pieces : 0, b->gen ? b->gen_ds_max : 0.0f, b->shared_weights);
    return;
  }
  launch_history_persist<R>(static_cast<const DevFault<R>*>(b->fs), b->chunks, b->nchunks, b->partial, b->mm, b->TM,
                            b->fc, b->shape, grid, ahead ? 2 : 1, st, ahead, b->gen ? b->wtab : nullptr,
                            b->gen ? b->gen_pieces : 0, b->gen ? b->gen_ds_max : 0.0f, b->bar, b->bar + 1,
                            b->bar_limit, static_cast<int>(b->members.size()), b->shared_weights);
}

// The groups' two passes as parallel branches of st (joined on st).
template <class R>
void batch_passes(sbiem_batch_s* b, cudaStream_t st, cudaEvent_t fork) {
  const size_t ng = b->groups.size();
  for (size_t k = 0; k < ng; ++k) {
    const auto& gr = b->groups[k];
    cudaStream_t bs = k == 0 ? st : b->branch[k - 1];
    if (k > 0) cudaStreamWaitEvent(bs, fork, 0);
    const DevFault<R>* fs = static_cast<const DevFault<R>*>(b->fs) + gr.first;
    launch_pass_batch<R>(gr.g, fs, gr.count, gr.N, 1, 1, bs);
    launch_pass_batch<R>(gr.g, fs, gr.count, gr.N, 2, 1, bs);
    if (k > 0) {
      cudaEventRecord(b->fork_join[k], bs);
      cudaStreamWaitEvent(st, b->fork_join[k], 0);
    }
  }
}

// One step of every member (dt_min).  Plain: whole-window sums, passes,
// commits.  Overlapped (every member's AT/AN already hold this step's sums):
// a side branch sweeps the next step's sums (BT/BN) while the groups'
// passes run; after the join the commits add each member's newest interval.
template <class R>
void batch_enqueue_step(sbiem_batch_s* b, cudaStream_t st) {
  const bool ov = b->overlap;
  if (!ov) batch_history<R>(b, st);
  cudaEventRecord(b->ev_fork, st);
  if (ov) {
    cudaStreamWaitEvent(b->side, b->ev_fork, 0);
    batch_history<R>(b, b->side, true);
    cudaEventRecord(b->ev_side, b->side);
  }
  batch_passes<R>(b, st, b->ev_fork);
  if (ov) cudaStreamWaitEvent(st, b->ev_side, 0);
  for (const auto& gr : b->groups)
    launch_commit_batch<R>(static_cast<const DevFault<R>*>(b->fs) + gr.first, gr.count, gr.N, 1, st, ov ? 0 : -1);
}

}  // namespace

extern "C" {

int sbiem_batch_create(sbiem_batch_t* out, int n, const sbiem_t* members, int64_t chunk_slots) {
  if (!out || n < 1 || !members) return fail(SBIEM_ERR_INVALID, "bad argument");
  *out = nullptr;
  const bool fp32 = members[0] && members[0]->fp32();
  for (int r = 0; r < n; ++r) {
    if (!members[r]) return fail(SBIEM_ERR_INVALID, "NULL member");
    if (members[r]->fp32() != fp32) return fail(SBIEM_ERR_INVALID, "batch members must share the precision");
    if (members[r]->device != members[0]->device) return fail(SBIEM_ERR_INVALID, "batch members on several devices");
    for (int q = 0; q < r; ++q)
      if (members[q] == members[r]) return fail(SBIEM_ERR_INVALID, "a member appears twice");
  }
  auto* b = new sbiem_batch_s();
  b->fp32 = fp32;
  // group by N (stable), groups in order of first appearance
  std::vector<int> Ns;
  for (int r = 0; r < n; ++r)
    if (std::find(Ns.begin(), Ns.end(), members[r]->N) == Ns.end()) Ns.push_back(members[r]->N);
  for (int Nv : Ns) {
    sbiem_batch_s::Group gr{};
    gr.N = Nv;
    gr.first = static_cast<int>(b->members.size());
    for (int r = 0; r < n; ++r)
      if (members[r]->N == Nv) {
        b->members.push_back(members[r]);
        b->order.push_back(r);
      }
    gr.count = static_cast<int>(b->members.size()) - gr.first;
    gr.g = fp32 ? make_geom(Nv, sizeof(float2)) : make_geom(Nv, sizeof(double2));
    if (fp32) configure_batch_kernels<float>(gr.g);
    else configure_batch_kernels<double>(gr.g);
    b->groups.push_back(gr);
  }
  for (int r = 1; r < n; ++r)
    if (members[r]->sweep_shape != members[0]->sweep_shape) {
      delete b;
      return fail(SBIEM_ERR_INVALID, "batch members must share the history sweep shape");
    }
  b->shape = members[0]->sweep_shape;
  if (chunk_slots > 0 && chunk_slots != members[0]->chunk_slots) {
    // another chunk length: the first sweep shape with chunks of that length
    int sh_ok = -1;
    for (int sh = 0; sh <= 4 && sh_ok < 0; ++sh)
      if (sweep_chunk_slots(fp32 ? 1 : 0, sh) == chunk_slots) sh_ok = sh;
    if (sh_ok < 0) {
      delete b;
      return fail(SBIEM_ERR_INVALID, "chunk_slots must be 0 or the chunk length of a sweep shape");
    }
    b->shape = sh_ok;
  }
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, members[0]->device);
  if (fp32) {
    // one weight table for all: the members' tables cover each its own s
    // range of one function when c_s/c_p and dt_min agree; take the widest
    bool same = true;
    const sbiem_s* widest = members[0];
    for (int r = 0; r < n; ++r) {
      const sbiem_s* m = members[r];
      same = same && m->f32.wtab && m->p.cs / m->p.cp == members[0]->p.cs / members[0]->p.cp &&
             m->dt_min == members[0]->dt_min;
      if (m->gen_pieces > widest->gen_pieces) widest = m;
    }
    if (same) {
      b->wtab = widest->f32.wtab;
      b->gen_pieces = widest->gen_pieces;
      b->gen = true;
      b->gen_ds_max = kGenDsMaxDefault;
    }
  }
  b->per_sm_plain = fp32 ? persist_blocks_per_sm<float>(b->shape, false) : persist_blocks_per_sm<double>(b->shape, false);
  b->per_sm_gen = b->gen ? persist_blocks_per_sm<float>(b->shape, true) : 0;
  if (b->per_sm_plain < 1) b->per_sm_plain = 1;
  if (b->per_sm_gen < 1) b->per_sm_gen = 1;
  b->per_sm = b->gen ? b->per_sm_gen : b->per_sm_plain;
  b->hist_grid = b->sm_count * b->per_sm;
  b->chunk_slots = chunk_slots > 0 ? chunk_slots : members[0]->chunk_slots;
  if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return fail(SBIEM_ERR_CUDA, "stream creation failed");
  }
  b->stream = b->own;
  b->branch.resize(b->groups.size() > 1 ? b->groups.size() - 1 : 0);
  for (auto& st : b->branch) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  b->fork_join.resize(b->groups.size());
  for (auto& e : b->fork_join) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&b->ev_side, cudaEventDisableTiming);
  {
    // the overlapped sweep leaves room for the one-launch FP32 passes
    bool small = fp32;
    for (auto* m : b->members) small = small && m->N <= kFusedMaxN;
    b->lag_grid = small ? b->sm_count : b->hist_grid;
  }
  for (auto* m : b->members) cudaStreamSynchronize(m->stream);
  int rc = fp32 ? batch_build<float>(b) : batch_build<double>(b);
  if (rc) {
    batch_free(b);
    delete b;
    return rc;
  }
  *out = b;
  return SBIEM_OK;
}

void sbiem_batch_destroy(sbiem_batch_t b) {
  if (!b) return;
  batch_free(b);
  delete b;
}

int sbiem_batch_set_stream(sbiem_batch_t b, void* stream) {
  if (!b) return fail(SBIEM_ERR_INVALID, "NULL batch");
  CK(cudaStreamSynchronize(b->stream));
  b->stream = stream ? static_cast<cudaStream_t>(stream) : cudaStreamLegacy;
  return SBIEM_OK;
}

int sbiem_batch_enqueue(sbiem_batch_t b, int64_t nsteps) {
  if (!b || nsteps < 0) return fail(SBIEM_ERR_INVALID, "bad argument");
  // overlapped: every member's AT/AN must hold the next step's sums (they do
  // after an overlapped sequence, batched or not, unless a member changed)
  bool valid = true;
  for (auto* m : b->members) valid = valid && m->lag_m == 1;
  if (b->overlap && !valid && nsteps > 0) {
    if (b->fp32) batch_history<float>(b, b->stream);
    else batch_history<double>(b, b->stream);
    CK(cudaGetLastError());
  }
  if (!b->graph) {
    CK(cudaStreamSynchronize(b->stream));
    CK(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal));
    if (b->fp32) batch_enqueue_step<float>(b, b->own);
    else batch_enqueue_step<double>(b, b->own);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamEndCapture(b->own, &b->graph_def);
    if (e1 != cudaSuccess || e2 != cudaSuccess)
      return fail(SBIEM_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    CK(cudaGraphInstantiate(&b->graph, b->graph_def, 0));
  }
  for (int64_t k = 0; k < nsteps; ++k) CK(cudaGraphLaunch(b->graph, b->stream));
  if (nsteps > 0)
    for (auto* m : b->members) m->lag_m = b->overlap ? 1 : -1;
  return SBIEM_OK;
}

int sbiem_batch_status(sbiem_batch_t b, uint32_t* flags, int64_t* steps_done) {
  if (!b) return fail(SBIEM_ERR_INVALID, "NULL batch");
  CK(cudaStreamSynchronize(b->stream));
  for (size_t q = 0; q < b->members.size(); ++q) {
    uint32_t fl = 0;
    int64_t sd = 0;
    int rc = sbiem_status(b->members[q], &fl, &sd, 0);
    if (rc) return rc;
    if (flags) flags[b->order[q]] = fl;
    if (steps_done) steps_done[b->order[q]] = sd;
  }
  return SBIEM_OK;
}

int sbiem_batch_set_wait_limit(sbiem_batch_t b, int64_t polls) {
  if (!b || polls < 0) return fail(SBIEM_ERR_INVALID, "NULL batch or negative limit");
  CK(cudaStreamSynchronize(b->stream));
  b->bar_limit = polls;
  if (b->graph) {
    // the step graph holds the old limit
    cudaGraphExecDestroy(b->graph);
    cudaGraphDestroy(b->graph_def);
    b->graph = nullptr;
    b->graph_def = nullptr;
  }
  return SBIEM_OK;
}

int sbiem_batch_get_sweep(sbiem_batch_t b, int32_t* shape, double* gen_ds_max, int32_t* ctas_per_sm,
                          int32_t* overlap, int32_t* distinct_weights, int32_t* persistent) {
  if (!b) return fail(SBIEM_ERR_INVALID, "NULL batch");
  if (shape) *shape = b->shape;
  if (gen_ds_max) *gen_ds_max = b->gen ? static_cast<double>(b->gen_ds_max) : 0.0;
  if (ctas_per_sm) *ctas_per_sm = b->hist_grid / (b->sm_count > 0 ? b->sm_count : 1);
  if (overlap) *overlap = b->overlap ? 1 : 0;
  if (distinct_weights) *distinct_weights = b->distinct_weights;
  if (persistent) *persistent = b->persistent ? 1 : 0;
  return SBIEM_OK;
}

int sbiem_batch_set_persistent(sbiem_batch_t b, int on, int* on_out) {
  if (!b || (on != 0 && on != 1)) return fail(SBIEM_ERR_INVALID, "bad argument");
  if (on_out) *on_out = b->persistent ? 1 : 0;
  if ((on == 1) == b->persistent) return SBIEM_OK;
  CK(cudaStreamSynchronize(b->stream));
  b->persistent = on == 1;
  if (b->graph) {
    // the step graph holds the other form
    cudaGraphExecDestroy(b->graph);
    cudaGraphDestroy(b->graph_def);
    b->graph = nullptr;
    b->graph_def = nullptr;
  }
  return SBIEM_OK;
}

int sbiem_batch_set_overlap(sbiem_batch_t b, int on, int* on_out) {
  if (!b || (on != 0 && on != 1)) return fail(SBIEM_ERR_INVALID, "bad argument");
  if (on_out) *on_out = b->overlap ? 1 : 0;
  if ((on == 1) == b->overlap) return SBIEM_OK;
  CK(cudaStreamSynchronize(b->stream));
  b->overlap = on == 1;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    cudaGraphDestroy(b->graph_def);
    b->graph = nullptr;
    b->graph_def = nullptr;
  }
  return SBIEM_OK;
}

int sbiem_batch_tune(sbiem_batch_t b, int reps, int64_t* chunk_out, int* blocks_out, float* ms_out) {
  if (!b || reps < 1) return fail(SBIEM_ERR_INVALID, "bad argument");
  // resident sweep CTAs per SM: 1 .. the occupancy limit; the chunk length
  // is the members' (their sweep shape)
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_b = b->hist_grid / b->sm_count;
  bool best_gen = b->gen;
  float best_thr = b->gen_ds_max;
  int best_shape = b->shape;
  const bool can_gen = b->wtab != nullptr;
  std::vector<float> thr = {0.0f};
  if (can_gen)
    for (double v : {kGenDsBlockMax / 4.0, kGenDsBlockMax, kGenDsBlock4Max}) thr.push_back(static_cast<float>(v));
  // the sweep shapes that keep the members' chunk length (their chunk
  // tables and per-mode chunk ranges stay valid)
  // every sweep shape, each with the ensemble's chunk table of its chunk
  // length (the mode-block size: 512, 1024 or 2048 lags in FP32)
  const int prec = b->fp32 ? 1 : 0;
  for (int sh = 0; sh <= 4; ++sh)
  for (float tv : thr) {
    {
      const int rc_ch = batch_use_chunks(b, sweep_chunk_slots(prec, sh));
      if (rc_ch) return rc_ch;
    }
    b->shape = sh;
    b->gen = tv > 0.0f;
    b->gen_ds_max = tv;
    const int lim = b->gen ? persist_blocks_per_sm<float>(sh, true)
                           : (b->fp32 ? persist_blocks_per_sm<float>(sh, false)
                                      : persist_blocks_per_sm<double>(sh, false));
    for (int bl = 1; bl <= lim; ++bl) {
      b->hist_grid = b->sm_count * bl;
      // one untimed launch, then reps timed ones; take the median
      if (b->fp32) batch_history<float>(b, b->stream);
      else batch_history<double>(b, b->stream);
      std::vector<float> t;
      for (int k = 0; k < reps; ++k) {
        CK(cudaEventRecord(e0, b->stream));
        if (b->fp32) batch_history<float>(b, b->stream);
        else batch_history<double>(b, b->stream);
        CK(cudaEventRecord(e1, b->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        t.push_back(ms);
      }
      std::sort(t.begin(), t.end());
      const float med = t[t.size() / 2];
      if (med < best) {
        best = med;
        best_b = bl;
        best_gen = b->gen;
        best_thr = tv;
        best_shape = sh;
      }
    }
  }
  b->shape = best_shape;
  {
    const int rc_ch = batch_use_chunks(b, sweep_chunk_slots(prec, best_shape));
    if (rc_ch) return rc_ch;
  }
  b->gen = best_gen;
  b->gen_ds_max = best_thr;
  b->per_sm_plain = b->fp32 ? persist_blocks_per_sm<float>(b->shape, false)
                            : persist_blocks_per_sm<double>(b->shape, false);
  b->per_sm_gen = b->gen ? persist_blocks_per_sm<float>(b->shape, true) : b->per_sm_gen;
  b->per_sm = b->gen ? b->per_sm_gen : b->per_sm_plain;
  b->hist_grid = b->sm_count * best_b;
  // The history form (one persistent launch or two launches; they agree
  // bitwise) and the overlap are chosen together: the cooperative launch
  // waits for room beside the passes, so which form is faster depends on the
  // overlap (256 members: 2.66 ms per step persistent without overlap, 2.42
  // ms two-launch with it).  Candidates: each form without overlap (its
  // sweep alone + the passes) and each form with overlap (its next-step
  // sweep and the passes timed together, for 1 .. (occupancy limit) sweep
  // CTAs per SM).  The passes write only staging arrays, so timing them
  // leaves the committed state alone; the status words they may set are put
  // back.  Nine timed launches at least per candidate: the totals are close.
  {
    const int reps_ov = std::max(reps, 9);
    auto timed = [&](auto&& launch, float* out) -> int {
      launch();
      std::vector<float> t;
      for (int k = 0; k < reps_ov; ++k) {
        CK(cudaEventRecord(e0, b->stream));
        launch();
        CK(cudaEventRecord(e1, b->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        t.push_back(ms);
      }
      std::sort(t.begin(), t.end());
      *out = t[t.size() / 2];
      return SBIEM_OK;
    };
    std::vector<unsigned> st0(b->members.size());
    for (size_t r = 0; r < b->members.size(); ++r)
      CK(cudaMemcpyAsync(&st0[r], b->members[r]->f64.status, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    float t_pass = 0.f;
    int rc = timed([&] {
      cudaEventRecord(b->ev_fork, b->stream);
      if (b->fp32) batch_passes<float>(b, b->stream, b->ev_fork);
      else batch_passes<double>(b, b->stream, b->ev_fork);
    }, &t_pass);
    if (rc) return rc;
    const int lim = b->gen ? persist_blocks_per_sm<float>(b->shape, true)
                           : (b->fp32 ? persist_blocks_per_sm<float>(b->shape, false)
                                      : persist_blocks_per_sm<double>(b->shape, false));
    float t_best = 1e30f, t_sweep_kept = best;
    bool ov_best = false, pers_best = true;
    int lag_best = b->lag_grid;
    for (int form = 0; form < 2; ++form) {
      b->persistent = form == 1;
      float t_sw = 0.f;
      rc = timed([&] {
        if (b->fp32) batch_history<float>(b, b->stream);
        else batch_history<double>(b, b->stream);
      }, &t_sw);
      if (rc) return rc;
      if (t_sw + t_pass < t_best) {
        t_best = t_sw + t_pass;
        ov_best = false;
        pers_best = b->persistent;
        t_sweep_kept = t_sw;
      }
      for (int lc = 1; lc <= std::max(1, lim); ++lc) {
        b->lag_grid = b->sm_count * lc;
        float t = 0.f;
        rc = timed([&] {
          cudaEventRecord(b->ev_fork, b->stream);
          cudaStreamWaitEvent(b->side, b->ev_fork, 0);
          if (b->fp32) batch_history<float>(b, b->side, true);
          else batch_history<double>(b, b->side, true);
          cudaEventRecord(b->ev_side, b->side);
          if (b->fp32) batch_passes<float>(b, b->stream, b->ev_fork);
          else batch_passes<double>(b, b->stream, b->ev_fork);
          cudaStreamWaitEvent(b->stream, b->ev_side, 0);
        }, &t);
        if (rc) return rc;
        if (t < t_best) {
          t_best = t;
          ov_best = true;
          pers_best = b->persistent;
          lag_best = b->lag_grid;
          t_sweep_kept = t_sw;
        }
      }
    }
    b->persistent = pers_best;
    b->overlap = ov_best;
    b->lag_grid = lag_best;
    best = t_sweep_kept;
    for (size_t r = 0; r < b->members.size(); ++r)
      CK(cudaMemcpyAsync(b->members[r]->f64.status, &st0[r], sizeof(unsigned), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the step graph holds the old grid
  CK(cudaStreamSynchronize(b->stream));
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    cudaGraphDestroy(b->graph_def);
    b->graph = nullptr;
    b->graph_def = nullptr;
  }
  if (chunk_out) *chunk_out = b->chunk_slots;
  if (blocks_out) *blocks_out = best_b;
  if (ms_out) *ms_out = best;
  return SBIEM_OK;
}

}  // extern "C"

// ------------------------------------------------------------- checkpoints
namespace {

constexpr char kCkMagic[8] = {'S', 'B', 'I', 'E', 'M', 'C', 'K', '3'};

struct CkHeader {
  char magic[8];
  int64_t N, total_slots;
  int32_t precision, state_law, kc_units, newton_maxit, quadrature, reserved;
  double dx, mu, cs, cp, beta_min, eta_w, kc_L, newton_tol, f0, V0, kcN_L;
};

// Element arrays of a checkpoint, in file order: inputs, then raw state.
std::vector<double*> ck_element_arrays(sbiem_s* s) {
  auto& f = s->f64;
  return {f.kappa, f.a, f.b, f.Dc, f.sig0, f.tau0, f.taur, f.Vp, f.V, f.xV, f.psi, f.th, f.thd, f.delta};
}

}  // namespace

extern "C" {

int sbiem_get_params(sbiem_t s, sbiem_params* out) {
  if (!s || !out) return fail(SBIEM_ERR_INVALID, "NULL argument");
  *out = s->p;
  return SBIEM_OK;
}

int sbiem_save(sbiem_t s, const char* path) {
  if (!s || !path) return fail(SBIEM_ERR_INVALID, "NULL argument");
  const int N = s->N;
  const auto& f = s->f64;
  CkHeader hd{};
  std::memcpy(hd.magic, kCkMagic, 8);
  hd.N = N;
  hd.total_slots = s->total_slots;
  hd.precision = s->p.precision;
  hd.state_law = s->p.state_law;
  hd.kc_units = s->p.kc_units;
  hd.newton_maxit = s->p.newton_maxit;
  hd.quadrature = s->p.quadrature;
  hd.dx = s->p.dx;
  hd.mu = s->p.mu;
  hd.cs = s->p.cs;
  hd.cp = s->p.cp;
  hd.beta_min = s->p.beta_min;
  hd.eta_w = s->p.eta_w;
  hd.kc_L = s->p.kc_L;
  hd.kcN_L = s->p.kcN_L;
  hd.newton_tol = s->p.newton_tol;
  hd.f0 = s->p.f0;
  hd.V0 = s->p.V0;
  const auto arrs = ck_element_arrays(s);
  std::vector<double> el(arrs.size() * static_cast<size_t>(N));
  std::vector<uint8_t> pr(N);
  std::vector<double2> spec(2 * static_cast<size_t>(s->nmodes));
  std::vector<int32_t> heads(s->nmodes);
  const size_t slot = s->fp32() ? sizeof(Slot32) : sizeof(Slot64);
  std::vector<unsigned char> ring(slot * static_cast<size_t>(s->total_slots));
  double t = 0.0;
  long long steps = 0;
  for (size_t k = 0; k < arrs.size(); ++k)
    CK(cudaMemcpyAsync(el.data() + k * N, arrs[k], sizeof(double) * N, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(pr.data(), f.presc, N, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(spec.data(), f.dhat, sizeof(double2) * s->nmodes, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(spec.data() + s->nmodes, f.khat, sizeof(double2) * s->nmodes, cudaMemcpyDeviceToHost,
                     s->stream));
  CK(cudaMemcpyAsync(heads.data(), f.head, sizeof(int32_t) * s->nmodes, cudaMemcpyDeviceToHost, s->stream));
  const void* ring_dev = s->fp32() ? static_cast<const void*>(s->f32.ring) : static_cast<const void*>(s->f64.ring);
  if (!ring.empty()) CK(cudaMemcpyAsync(ring.data(), ring_dev, ring.size(), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(&t, f.t, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(&steps, f.steps_done, sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(SBIEM_ERR_INVALID, std::string("cannot open ") + path);
  bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1 && std::fwrite(el.data(), sizeof(double), el.size(), fp) == el.size() &&
            std::fwrite(pr.data(), 1, pr.size(), fp) == pr.size() &&
            std::fwrite(spec.data(), sizeof(double2), spec.size(), fp) == spec.size() &&
            std::fwrite(heads.data(), sizeof(int32_t), heads.size(), fp) == heads.size() &&
            std::fwrite(ring.data(), 1, ring.size(), fp) == ring.size() && std::fwrite(&t, sizeof(t), 1, fp) == 1 &&
            std::fwrite(&steps, sizeof(steps), 1, fp) == 1;
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok) return fail(SBIEM_ERR_INVALID, std::string("write failed: ") + path);
  // the next step recomputes its history sums, as a loaded handle does, so
  // the two continue identically (the overlapped form sums in another order)
  s->lag_m = -1;
  return SBIEM_OK;
}

}  // extern "C"

namespace {

// Every check of a checkpoint that needs no device: the header's
// parameters, the history size they imply and each mode's ring head.  On
// success *hd holds the header and the file is positioned after it.
int load_checked(FILE* fp, const char* path, CkHeader* hd_out, sbiem_params* p_out, std::vector<int64_t>* R_out) {
  CkHeader hd{};
  if (std::fread(&hd, sizeof(hd), 1, fp) != 1 || std::memcmp(hd.magic, kCkMagic, 8) != 0 || !is_pow2(hd.N) ||
      hd.N < 16 || hd.N > (1 << 20) || hd.total_slots < 0)
    return fail(SBIEM_ERR_INVALID, std::string("not a checkpoint: ") + path);
  sbiem_params p;
  sbiem_default_params(&p);
  p.N = hd.N;
  p.precision = hd.precision;
  p.state_law = hd.state_law;
  p.kc_units = hd.kc_units;
  p.newton_maxit = hd.newton_maxit;
  p.quadrature = hd.quadrature;
  p.dx = hd.dx;
  p.mu = hd.mu;
  p.cs = hd.cs;
  p.cp = hd.cp;
  p.beta_min = hd.beta_min;
  p.eta_w = hd.eta_w;
  p.kc_L = hd.kc_L;
  p.kcN_L = hd.kcN_L;
  p.newton_tol = hd.newton_tol;
  p.f0 = hd.f0;
  p.V0 = hd.V0;
  if (!(p.dx > 0) || !(p.cs > 0) || !(p.cp > p.cs) || !(p.beta_min > 0) || !(p.eta_w >= 0) || !(p.kc_L > 0) ||
      !(p.kcN_L >= 0) || (p.precision != 0 && p.precision != 1) || (p.kc_units != 0 && p.kc_units != 1) ||
      (p.quadrature != 0 && p.quadrature != 1) ||
      !std::isfinite(p.dx * p.cs * p.cp * p.beta_min * p.eta_w * p.kc_L * p.kcN_L))
    return fail(SBIEM_ERR_INVALID, std::string("checkpoint parameters out of range: ") + path);
  // the history size the parameters imply, before any buffer is sized from the file
  const double L = static_cast<double>(p.N) * p.dx, dt_min = p.beta_min * p.dx / p.cs;
  const double longest = p.eta_w * L / p.cs / dt_min;
  if (!(longest < 2.0e9)) return fail(SBIEM_ERR_INVALID, std::string("checkpoint windows too long: ") + path);
  std::vector<int64_t> M, MT, MN;
  windows(p, L, dt_min, M, MT, MN);
  int64_t total = 0;
  R_out->assign(M.size(), 0);
  for (size_t n = 0; n < M.size(); ++n) {
    (*R_out)[n] = std::max<int64_t>(M[n] - 1, 0);
    total += (*R_out)[n];
  }
  if (total != hd.total_slots)
    return fail(SBIEM_ERR_INVALID, "checkpoint history size does not match its parameters: " + std::string(path));
  *hd_out = hd;
  *p_out = p;
  return SBIEM_OK;
}

}  // namespace

static int sbiem_load_body(sbiem_t* out, const char* path, const sbiem_params* alloc) {
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(SBIEM_ERR_INVALID, std::string("cannot open ") + path);
  CkHeader hd{};
  sbiem_params p;
  std::vector<int64_t> Rn;
  const int rc0 = load_checked(fp, path, &hd, &p, &Rn);
  if (rc0 != SBIEM_OK) {
    std::fclose(fp);
    return rc0;
  }
  const int N = static_cast<int>(hd.N);
  const size_t nm = static_cast<size_t>(N / 2 + 1);
  const size_t n_el = 14;
  std::vector<double> el(n_el * static_cast<size_t>(N));
  std::vector<uint8_t> pr(N);
  std::vector<double2> spec(2 * nm);
  std::vector<int32_t> heads(nm);
  const size_t slot = hd.precision == 1 ? sizeof(Slot32) : sizeof(Slot64);
  std::vector<unsigned char> ring(slot * static_cast<size_t>(hd.total_slots));
  double t = 0.0;
  long long steps = 0;
  bool ok = std::fread(el.data(), sizeof(double), el.size(), fp) == el.size() &&
            std::fread(pr.data(), 1, pr.size(), fp) == pr.size() &&
            std::fread(spec.data(), sizeof(double2), spec.size(), fp) == spec.size() &&
            std::fread(heads.data(), sizeof(int32_t), heads.size(), fp) == heads.size() &&
            std::fread(ring.data(), 1, ring.size(), fp) == ring.size() && std::fread(&t, sizeof(t), 1, fp) == 1 &&
            std::fread(&steps, sizeof(steps), 1, fp) == 1;
  std::fclose(fp);
  if (!ok) return fail(SBIEM_ERR_INVALID, std::string("truncated checkpoint: ") + path);
  // ring heads index the sweep's copies: 0 <= head_n < R_n (0 where a mode has no history)
  for (size_t n = 0; n < nm; ++n)
    if (heads[n] < 0 || (Rn[n] > 0 ? heads[n] >= Rn[n] : heads[n] != 0))
      return fail(SBIEM_ERR_INVALID, "checkpoint ring head out of range at mode " + std::to_string(n));
  if (alloc) {
    p.alloc_fn = alloc->alloc_fn;
    p.free_fn = alloc->free_fn;
    p.alloc_user = alloc->alloc_user;
  }
  auto arr = [&](int k) { return el.data() + static_cast<size_t>(k) * N; };
  // inputs in file order: kappa, a, b, Dc, sigma_load, tau_load, tau_rate, V_presc;
  // state: V, xV, psi, theta, thetadot, delta
  bool any_pr = false;
  for (int i = 0; i < N; ++i) any_pr = any_pr || pr[i];
  sbiem_t s = nullptr;
  int rc = sbiem_create(&s, &p, nullptr, arr(0), arr(1), arr(2), arr(3), arr(4), arr(5), arr(6),
                        any_pr ? pr.data() : nullptr, any_pr ? arr(7) : nullptr, arr(8), arr(11));
  if (rc) return rc;
  if (static_cast<int64_t>(s->total_slots) != hd.total_slots) {
    sbiem_destroy(s);
    return fail(SBIEM_ERR_INVALID, "checkpoint history size does not match its parameters");
  }
  auto& f = s->f64;
  double* raw[] = {f.V, f.xV, f.psi, f.th, f.thd, f.delta};
  auto fail_cuda = [&](cudaError_t e) {
    sbiem_destroy(s);
    return fail(SBIEM_ERR_CUDA, std::string("load: ") + cudaGetErrorString(e));
  };
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 6 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(raw[k], arr(8 + k), sizeof(double) * N, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f.dhat, spec.data(), sizeof(double2) * nm, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f.khat, spec.data() + nm, sizeof(double2) * nm, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f.head, heads.data(), sizeof(int32_t) * nm, cudaMemcpyHostToDevice, s->stream);
  void* ring_dev = s->fp32() ? static_cast<void*>(s->f32.ring) : static_cast<void*>(s->f64.ring);
  if (e == cudaSuccess && !ring.empty())
    e = cudaMemcpyAsync(ring_dev, ring.data(), ring.size(), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f.t, &t, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f.steps_done, &steps, sizeof(long long), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && f.dhat32) {
    launch_to_float2(f.dhat, f.dhat32, s->nmodes, s->stream);
    launch_to_float2(f.khat, f.khat32, s->nmodes, s->stream);
  }
  if (e == cudaSuccess && s->f32.zin1) launch_zin(f.V, f.kappa, s->f32.zin1, s->N, s->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return fail_cuda(e);
  s->lag_m = -1;
  *out = s;
  return SBIEM_OK;
}

extern "C" int sbiem_load(sbiem_t* out, const char* path, const sbiem_params* alloc) {
  if (!out || !path) return fail(SBIEM_ERR_INVALID, "NULL argument");
  *out = nullptr;
  try {
    return sbiem_load_body(out, path, alloc);
  } catch (const std::exception& ex) {
    // host buffers sized from a corrupt file (already bounded above) or any
    // other host failure: an error code, never an exception across the C ABI
    return fail(SBIEM_ERR_INVALID, std::string("checkpoint load failed: ") + ex.what());
  }
}
