// Device types, launch descriptors and host-side launch wrappers of libsbiem.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "mlp.cuh"
#include "sbiem.h"

namespace sbiem {

// ------------------------------------------------------------ complex types
template <class R> struct CxT;
template <> struct CxT<double> { using T = double2; };
template <> struct CxT<float> { using T = float2; };
template <class R> using Cx = typename CxT<R>::T;

// One history slot of one mode: F[Vbar] (shear field) and F[kappa Vbar]
// (normal field), complex each.
struct __align__(32) Slot64 { double2 t, n; };
using Slot32 = float4;  // (T.re, T.im, N.re, N.im)
template <class R> struct SlotT;
template <> struct SlotT<double> { using T = Slot64; };
template <> struct SlotT<float> { using T = Slot32; };
template <class R> using Slot = typename SlotT<R>::T;

// Entries per mode of the current-interval weight table (m = 2^p, p < 41).
constexpr int kPow2Slots = 41;

// Kernel weight pair (w^T_{n,j}, w^N_{n,j}) of one lag.
template <class R> using W2 = Cx<R>;

// One chunk of consecutive history slots of one mode.
struct Chunk {
  int32_t mode;
  int32_t first;  // chunk index of the mode's first chunk
  int32_t count;  // chunks of this mode
  int32_t pad;    // ensemble member (batched history convolution), else 0
  int64_t i0, i1;  // slot range [i0, i1) within the mode's ring
};


// Four-step FFT geometry: N = N1 * N2, column pass (length N2) then row pass
// (length N1); B columns or rows per CTA.
struct FftGeom {
  int N, N1, N2, lgN1, lgN2, Bc, Br, tc, tr;
};

// Pointers of one fault on the device.
template <class R>
struct DevFault {
  using Real = R;
  int N;
  int nmodes;          // N/2 + 1
  double L, S, mu, eta, reta, dt_min, f0, V0, lnV0;  // reta = 1/eta
  int state_law;
  int newton_epw;                          // elements per Newton warp (1..32)
  int newton_maxit;
  double newton_tol;
  // element state (FP64)
  double *V, *psi, *thd, *delta;          // committed (psi = ln theta)
  double *th, *th2;                        // theta: committed, pass-2 (staged)
  double *V1, *thd1;                       // pass-1 results
  double *Vbar;                            // pass slip rate
  double *V2, *psi2, *thd2, *delta2;       // pass-2 results (staged)
  double *xV, *x1, *x2;                    // ln V: committed, pass 1, staged
  double *a, *b, *Dc, *sig0, *tau0, *taur, *Vp, *kappa;
  double *lvd;                             // ln(V0 / Dc) per element
  double *rDc;                             // 1 / Dc per element
  uint8_t* presc;
  // spectral state (FP64)
  double2 *dhat, *khat;                    // F[delta], F[kappa delta]
  double2 *U2, *Q2;                        // staged pass-2 spectra
  double2 *AT, *AN;                        // history sums
  double2 *BT, *BN;                        // next step's sums without its newest interval (overlapped form)
  double4* partial;                        // per-chunk partial sums
  int* counter;                            // per-mode chunk counters
  // history
  Slot<R>* ring;
  W2<R>* w;
  double2* w0pow;                          // [mode][p]: sum of the first 2^p weights
  float2* c0pow;                           // [mode][p]: S 2^p dt_min + mu w0 (T, N), FP32 form
  float2 *dhat32, *khat32, *AT32, *AN32;   // FP32 copies for the fused FP32 spectral kernel
  float2 *zin1, *zin2;                     // fused FP32 form: FFT inputs (Vbar, kappa Vbar) of passes 1, 2
  float2 *U2f, *Q2f;                       // fused FP32 form: staged pass-2 spectra
  const int64_t *ring_off, *w_off;
  const int32_t *Rn, *Mn;
  int32_t* head;
  const Chunk* chunks;
  int nchunks;
  const int32_t *mfirst, *mcount;          // per mode: first chunk, chunks
  int sweep_shape;                         // chunk length x stages of the history sweep (0..3)
  int lag_shape;                           // the same for the sweep beside the passes (0..4)
  // FP32 sweep with the weights evaluated on chip instead of streamed:
  // per mode (ds_hi, ds_lo, M^T bits, M^N bits) with ds = c_s k_n dt_min as
  // a two-float sum, and the piecewise-polynomial table of dt C(s)
  long long spin_limit;                    // polls of the sweep's consumer waits before it gives up
  float gen_ds_max;                        // modes with ds <= this evaluate their weights on chip,
                                           // the others stream them (0: every mode streams)
  const float4* wgen;
  const float4* wtab;                      // kGenPairs / 2 float4 per piece
  int wtab_pieces;
  // FFT work
  Cx<R> *z, *zt, *Z, *y;                   // natural-order input, transposed, spectrum, output
  const Cx<R>* tw;                         // exp(-2 pi i j/N)
  FftGeom g;
  // bookkeeping
  unsigned* status;
  long long* steps_done;
  double* t;
  unsigned long long* it_sum;
  int* it_max;
  unsigned long long* it_total;            // [iterations, solves] since the last reset
  const MlpDev* mlp;                       // Newton initial-guess network (NULL: off)
  float* harvest;                          // rows (ln V_prev, ln theta, tau/sigma, a, b, ln V*)
  unsigned long long* harvest_count;
  long long harvest_cap;
  int* work;                               // next chunk of the history convolution
};

// One-launch FP32 spectral pass: a single CTA of N/8 threads below
// kClusterMinN, a cluster of cluster_ctas(N) CTAs from kClusterMinN to
// kFusedMaxN; larger N use the four-kernel path.
constexpr int kFusedMaxN = 16384;
constexpr int kClusterMinN = 2048;
constexpr int kClusterCTAs = 8;
// CTAs per cluster for a given N: 16 (a non-portable cluster size) from
// N = 4096: half the work per CTA on the latency-bound pass (flushed steps
// without history at N = 4096: 35.3 -> 33.0 us; N = 8192: 49.2 -> 36.9 us;
// at N = 2048 it lost, 39.4 -> 40.9 us with history), and at N = 16384 half
// the per-CTA shared memory, so the pass fits beside a history-sweep CTA.
__host__ __device__ constexpr int cluster_ctas(int N) { return N >= 4096 ? 16 : kClusterCTAs; }
// The same for the batched pass of an ensemble (one cluster per member, many
// clusters at once, beside the overlapped sweep): 8 below N = 16384, where
// clusters of 16 were slower (256 members: 2.42 against 2.76 ms per step).
__host__ __device__ constexpr int batch_cluster_ctas(int N) { return N >= 16384 ? 16 : kClusterCTAs; }
// Values per thread in each FFT stage of the cluster pass (4: radix-4
// stages, 8: radix-8 stages with half the threads).
#ifndef SBIEM_CLUSTER_EPT
#define SBIEM_CLUSTER_EPT 4
#endif
constexpr int kClusterEPT = SBIEM_CLUSTER_EPT;

// Host launch wrappers (kernels.cu).
// Plain streaming read of `bytes` (16-byte aligned; sbiem_read_probe).
void launch_read_probe(const void* p, int64_t bytes, float* sink, int sm_count, cudaStream_t st);
// History sums AT/AN of a step of m_dt (bulk-async sweep, then per-mode
// sums of its chunk partials).
template <class R> void launch_history(const DevFault<R>& f, int m_dt, int grid, cudaStream_t st,
                                       cudaEvent_t sweep_done = nullptr);
// The one-warp-per-chunk sweep with atomic chunk hand-out and per-mode
// last-arriver sums (writes AT/AN itself); used on caller-owned buffers.
template <class R> void launch_history_atomic(const DevFault<R>& f, int m_dt, int grid, cudaStream_t st);
// Resident CTAs per SM of the bulk-async sweep (gen: the form that can
// evaluate weights on chip); its chunk length.
template <class R> int sweep_blocks_per_sm(int shape, bool gen = false);
int sweep_chunk_slots(int precision, int shape);
// The same sweep with the weights shifted by 2 m_dt, chunk partials only:
// the part of the next step's sums that does not involve this step's
// interval, computed while this step's passes run (overlapped form); the
// commit adds them up.
template <class R> void launch_history_ahead(const DevFault<R>& f, int m_dt, int grid, cudaStream_t st);
// Ensemble launches: fs is a device array of member descriptors; the pass and
// commit kernels take one member per blockIdx.y (all members of equal N).
// Ensemble history sums: one bulk-async sweep over the ensemble's chunk
// table (every member's modes in order, member in Chunk::pad), then per
// (member, mode) pair mm[t] the sum of its chunks [fc[t].x, fc[t].x +
// fc[t].y) into the member's AT/AN.
// wtab (FP32 only, or NULL): the members' shared on-chip weight table of
// wtab_pieces pieces (every member's wgen must then be set); modes with
// ds <= gen_ds_max evaluate their weights from it.
template <class R> void launch_history_batch(const DevFault<R>* fs, const Chunk* chunks, int nchunks,
                                             double4* partial, const int2* mm, int TM, const int2* fc,
                                             int shape, int grid, int m_dt, cudaStream_t st, bool ahead,
                                             const float4* wtab = nullptr, int wtab_pieces = 0,
                                             float gen_ds_max = 0.0f, bool ring_evict_first = false);
// The same as one persistent cooperative launch: the sweep, a grid barrier
// (counter and epoch in device memory, polled at most bar_limit times; on
// the limit every one of the `members` members is flagged SBIEM_FLAG_WAIT),
// then every (member, mode) sum.  grid must not exceed the resident CTAs
// (persist_blocks_per_sm x SMs).  ring_evict_first: ring slots are copied
// under an L2 evict-first policy (members share their weight runs, which
// then stay in L2).
template <class R> void launch_history_persist(const DevFault<R>* fs, const Chunk* chunks, int nchunks,
                                               double4* partial, const int2* mm, int TM, const int2* fc,
                                               int shape, int grid, int m_dt, cudaStream_t st, bool ahead,
                                               const float4* wtab, int wtab_pieces, float gen_ds_max,
                                               unsigned* bar_count, unsigned* bar_epoch, long long bar_limit,
                                               int members, bool ring_evict_first);
template <class R> int persist_blocks_per_sm(int shape, bool gen);
// Save (dir 0) or restore (dir 1) the ring slot of each mode that a step of
// one dt_min overwrites (buf: nmodes slots).
template <class R> void launch_slot_swap(const DevFault<R>& f, void* buf, int dir, cudaStream_t st);
template <class R> void launch_pass_batch(const FftGeom& g, const DevFault<R>* fs, int members, int N, int pass,
                                          int m_dt, cudaStream_t st);
template <class R> void launch_commit_batch(const DevFault<R>* fs, int members, int N, int m_dt, cudaStream_t st,
                                            int lag_p = -1);
template <class R> void configure_batch_kernels(const FftGeom& g);
// Resident CTAs per SM of the history convolution (occupancy calculator).
template <class R> int history_blocks_per_sm();
template <class R> void launch_pass(const DevFault<R>& f, int pass, int m_dt, cudaStream_t st);
// The two halves of launch_pass: the spectral kernels, then Newton (early).
// started (may be null): an event that fires once every CTA of the pass's
// first kernel has started.
template <class R> void launch_spectral(const DevFault<R>& f, int pass, int m_dt, cudaStream_t st,
                                        cudaEvent_t started = nullptr);
template <class R> void launch_newton(const DevFault<R>& f, int pass, int m_dt, cudaStream_t st);
// lag_p >= 0 (m_dt = 2^lag_p): also finish the next step's history sums,
// AT = BT + (sum of the weights of lags m_dt .. 2 m_dt - 1) x the new slot.
template <class R> void launch_commit(const DevFault<R>& f, int m_dt, cudaStream_t st, int lag_p = -1);
// Multi-slot history push for steps of m_dt > 1 (before launch_commit).
template <class R> void launch_push_multi(const DevFault<R>& f, int m_dt, cudaStream_t st);
// Fill f.w0pow from the weights (and f.c0pow when present).
template <class R> void launch_weight_pow2(const DevFault<R>& f, cudaStream_t st);
// FP32 copies of the spectral running sums (after they are recomputed).
void launch_to_float2(const double2* a, float2* out, int n, cudaStream_t st);
// zin1 = (V, kappa V) in FP32: the pass-1 input of the fused FP32 form
// (after V changes outside a committed step).
void launch_zin(const double* V, const double* kappa, float2* zin, int n, cudaStream_t st);
// Save (dir 0) / restore (dir 1) the ring slots a push of m_dt copies overwrites.
template <class R> void launch_ring_undo(const DevFault<R>& f, int m_dt, void* undo, int dir, cudaStream_t st);
// Ring slots ring[i] = (hT[i], hN[i]) from interleaved complex device arrays
// (FP32 when in_f32, else FP64), n slots.
template <class R> void launch_set_ring(Slot<R>* ring, const void* hT, const void* hN, bool in_f32, int64_t n,
                                        int sm_count, cudaStream_t st);
// *out = max_i |a_i - b_i|.
void launch_maxdiff(const double* a, const double* b, int n, double* out, cudaStream_t st);
// Weights of every lag from the Chebyshev table: quadrature 0 midpoint,
// 1 the integral over each interval.
template <class R> void launch_weights(const DevFault<R>& f, const double* cheb, int npieces, int deg,
                                       double h, double cs, const int32_t* MT, const int32_t* MN,
                                       int quadrature, cudaStream_t st);

// FP64 utility transforms on caller buffers of length N (natural order):
// forward: Z = sum_i z_i exp(-2 pi i n i/N); inverse: z = (1/N) sum_n Z_n exp(+...).
void launch_fft64(const FftGeom& g, const double2* tw, const double2* in, double2* tmp,
                  double2* out, bool inverse, cudaStream_t st);
// Pack z = x + i y from two real arrays; y may be NULL (zero imaginary part).
void launch_pack(int N, const double* x, const double* y, const double* ymul, double2* z, cudaStream_t st);
// From the spectrum Z of z = x + i y: X_n, Y_n for n = 0..N/2.
void launch_unpack(int N, const double2* Z, double2* X, double2* Y, cudaStream_t st);
// Z_n *= -k_{|n|}^2 (second derivative on the periodic grid of length L).
void launch_d2(int N, double L, double2* Z, cudaStream_t st);
void launch_real_part(int N, const double2* z, double* x, cudaStream_t st);

FftGeom make_geom(int N, int elem_bytes);
// Opt the FFT kernels into the dynamic shared memory they need (once per geometry).
template <class R> void configure_kernels(const FftGeom& g);

}  // namespace sbiem
