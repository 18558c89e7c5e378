// sm_103a kernels of the non-planar spectral BIEM time step (Sec. 3.3).
//
//   k_history  truncated history convolution A^X_n = sum_j w^X_{n,j} H^X_n
//              (Sec. 3.1, Sec. 3.3 step (2)), the bandwidth-bound hot loop
//   k_col      column pass of the four-step FFT; forward with the predictor
//              prologue (Vbar, kappa Vbar), inverse with the spectral
//              assembly prologue (static + current-interval + history terms)
//   k_row      row pass of the four-step FFT
//   k_newton   per-element state update and Newton solve of Eq. (momentum)
//              with radiation damping (Sec. 3.3 step (3))
//   k_commit   accept the step: state, spectral running sums, history push
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "kernels.cuh"
#include <math_constants.h>

namespace sbiem {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// --------------------------------------------------------- complex helpers
template <class C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// Programmatic dependent launch: a kernel launched with the programmatic
// serialization attribute may start while its predecessor runs; it must
// read nothing the predecessor chain writes before pdl_wait() returns.
// pdl_trigger() lets this kernel's own dependent start launching.  Both are
// no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Shared-memory address of a generic pointer into this CTA's shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// --------------------------------------------------------- shared-memory FFT
// B independent radix-2 Stockham (decimation in frequency, self-sorting)
// transforms of length M = 2^lgM on buf[b * M + i].  twm[j] = exp(-2 pi i j/M),
// j < M/2.  Each stage reads every butterfly into registers, synchronizes,
// then writes, so one buffer suffices.
constexpr int kMaxBfly = 8;

template <class C, bool INV>
__device__ void fft_batch(C* buf, int lgM, int B, const C* twm, int tid, int nth) {
  const int M = 1 << lgM;
  const int half = M >> 1;
  const int total = B * half;
  int lgs = 0;
  for (int lgn = lgM; lgn >= 1; --lgn, ++lgs) {
    const int s = 1 << lgs;
    const int m = 1 << (lgn - 1);
    C ra[kMaxBfly], rb[kMaxBfly];
#pragma unroll
    for (int k = 0; k < kMaxBfly; ++k) {
      const int beta = tid + k * nth;
      if (beta < total) {
        const int col = beta >> (lgM - 1);
        const int bb = beta & (half - 1);
        const int p = bb >> lgs;
        const int q = bb & (s - 1);
        const C* base = buf + col * M;
        const C a = base[q + s * p];
        const C c = base[q + s * (p + m)];
        C w = twm[p * s];
        if (INV) w.y = -w.y;
        ra[k] = cadd(a, c);
        rb[k] = cmul(csub(a, c), w);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kMaxBfly; ++k) {
      const int beta = tid + k * nth;
      if (beta < total) {
        const int col = beta >> (lgM - 1);
        const int bb = beta & (half - 1);
        const int p = bb >> lgs;
        const int q = bb & (s - 1);
        C* base = buf + col * M;
        base[q + s * (2 * p)] = ra[k];
        base[q + s * (2 * p + 1)] = rb[k];
      }
    }
    __syncthreads();
  }
}

enum { PRO_LOAD = 0, PRO_PASS = 1, PRO_ASSEMBLE = 2 };

// Spectral assembly of mode m = min(n, N-n) (Sec. 3.1, Sec. 3.3 step (2)):
//   U = F[Vbar], Q = F[kappa Vbar] from the packed spectrum Z of Vbar + i kappa Vbar,
//   tau_m = -|k| [ S (Dhat + dt U) + mu (w0T U + AT) ]
//   sig_m = -i sgn(k) [ S (Khat + dt Q) + mu (w0N Q + AN) ]   (0 at m = 0, N/2)
// and Y_n = tau_n + i sig_n of the full spectrum (conjugates for n > N/2).
template <class R>
__device__ __forceinline__ Cx<R> assemble(const DevFault<R>& f, int n, int pass, int m_dt, double dt) {
  const int N = f.N;
  const int m = n <= (N >> 1) ? n : N - n;
  const Cx<R> Zm = f.Z[m];
  const Cx<R> Zc = f.Z[(N - m) & (N - 1)];
  double2 U, Q;
  U.x = 0.5 * (static_cast<double>(Zm.x) + static_cast<double>(Zc.x));
  U.y = 0.5 * (static_cast<double>(Zm.y) - static_cast<double>(Zc.y));
  Q.x = 0.5 * (static_cast<double>(Zm.y) + static_cast<double>(Zc.y));
  Q.y = -0.5 * (static_cast<double>(Zm.x) - static_cast<double>(Zc.x));
  double tr = 0.0, ti = 0.0, sr = 0.0, si = 0.0;
  if (m > 0) {
    const double k = kTwoPi * m / f.L;
    // current interval [0, m_dt dt_min]: sum of the first m_dt weights
    double w0T = 0.0, w0N = 0.0;
    if ((m_dt & (m_dt - 1)) == 0) {
      const double2 w0 = f.w0pow[static_cast<size_t>(m) * kPow2Slots + (31 - __clz(m_dt))];
      w0T = w0.x;
      w0N = w0.y;
    } else {
      const int lim = min(m_dt, f.Mn[m]);
      const int64_t wo = f.w_off[m];
      for (int j = 0; j < lim; ++j) {
        const W2<R> w = f.w[wo + j];
        w0T += static_cast<double>(w.x);
        w0N += static_cast<double>(w.y);
      }
    }
    const double2 D = f.dhat[m], K = f.khat[m], AT = f.AT[m], AN = f.AN[m];
    // the static term of the current interval and its instantaneous dynamic
    // term nearly cancel (C(k, 0) = -(1 - r^2)): combine their coefficients
    // first, S dt + mu w0, then multiply the spectrum
    const double cT = f.S * dt + f.mu * w0T, cN = f.S * dt + f.mu * w0N;
    tr = -k * (f.S * D.x + cT * U.x + f.mu * AT.x);
    // the Nyquist coefficient of a real sequence is real: keep its real part
    ti = (m < (N >> 1)) ? -k * (f.S * D.y + cT * U.y + f.mu * AT.y) : 0.0;
    if (m < (N >> 1)) {
      const double xr = f.S * K.x + cN * Q.x + f.mu * AN.x;
      const double xi = f.S * K.y + cN * Q.y + f.mu * AN.y;
      sr = xi;   // -i (xr + i xi)
      si = -xr;
    }
  }
  if (pass == 2 && n <= (N >> 1)) {
    f.U2[n] = U;
    f.Q2[n] = Q;
  }
  if (n > (N >> 1)) {
    ti = -ti;
    si = -si;
  }
  Cx<R> Y;
  Y.x = static_cast<R>(tr - si);
  Y.y = static_cast<R>(ti + sr);
  return Y;
}

// Per-mode inputs of the precision form's assembly: running sums F[delta],
// F[kappa delta], history sums, and the coefficients S dt + mu w0 (T, N) of
// the current interval (from the power-of-two table, or summed in FP64 for
// other step lengths; the near-cancelling combination is done in FP64).
struct ModeIn {
  float2 D, K, AT, AN, C;
};

__device__ __forceinline__ ModeIn load_mode_in(const DevFault<float>& f, int m, int m_dt, double dt) {
  ModeIn in;
  in.D = f.dhat32[m];
  in.K = f.khat32[m];
  in.AT = f.AT32[m];
  in.AN = f.AN32[m];
  if ((m_dt & (m_dt - 1)) == 0) {
    in.C = f.c0pow[static_cast<size_t>(m) * kPow2Slots + (31 - __clz(m_dt))];
  } else {
    double w0T = 0.0, w0N = 0.0;
    const int lim = min(m_dt, f.Mn[m]);
    for (int j = 0; j < lim; ++j) {
      const W2<float> w = f.w[f.w_off[m] + j];
      w0T += w.x;
      w0N += w.y;
    }
    in.C = make_float2(static_cast<float>(f.S * dt + f.mu * w0T), static_cast<float>(f.S * dt + f.mu * w0N));
  }
  return in;
}

// Assembly of the mode pair (m, N-m) of the precision form from the packed
// spectrum Zm = Z[m], Zc = Z[(N-m) mod N] of Vbar + i kappa Vbar (Sec. 3.1,
// Sec. 3.3 step (2)): returns Y[m] and Y[N-m] of tau_el + i sigma_el and, in
// pass 2, leaves U, Q of mode m for the commit.  FP32 products.
__device__ __forceinline__ void assemble_pair32(const DevFault<float>& f, int m, float2 Zm, float2 Zc, int pass,
                                                const ModeIn& in, float2* Ym, float2* Yc) {
  const int N = f.N, half = N >> 1;
  const float Ux = 0.5f * (Zm.x + Zc.x), Uy = 0.5f * (Zm.y - Zc.y);
  const float Qx = 0.5f * (Zm.y + Zc.y), Qy = -0.5f * (Zm.x - Zc.x);
  float tr = 0.f, ti = 0.f, sr = 0.f, si = 0.f;
  if (m > 0) {
    const float mu = static_cast<float>(f.mu);
    const float S = static_cast<float>(f.S);
    const float k = static_cast<float>(kTwoPi / f.L) * static_cast<float>(m);
    const float cT = in.C.x, cN = in.C.y;
    tr = -k * (S * in.D.x + cT * Ux + mu * in.AT.x);
    ti = (m < half) ? -k * (S * in.D.y + cT * Uy + mu * in.AT.y) : 0.f;
    if (m < half) {
      const float xr = S * in.K.x + cN * Qx + mu * in.AN.x;
      const float xi = S * in.K.y + cN * Qy + mu * in.AN.y;
      sr = xi;
      si = -xr;
    }
  }
  if (pass == 2) {
    f.U2f[m] = make_float2(Ux, Uy);
    f.Q2f[m] = make_float2(Qx, Qy);
  }
  // Y_m = tau_m + i sig_m; Y_{N-m} = conj(tau_m) + i conj(sig_m)
  *Ym = make_float2(tr - si, ti + sr);
  *Yc = make_float2(tr + si, -ti + sr);
}

// Precision-form assembly of one coefficient n of the full spectrum (the
// four-step passes): the pair (m, N-m), m = min(n, N-n), in FP32 from the
// FP32 per-mode inputs, Y[n] its half; U, Q of mode m are kept (pass 2) by
// the thread with n <= N/2.
__device__ __forceinline__ float2 assemble32_at(const DevFault<float>& f, int n, int pass, int m_dt, double dt) {
  const int N = f.N, half = N >> 1;
  const int m = n <= half ? n : N - n;
  const ModeIn in = load_mode_in(f, m, m_dt, dt);
  float2 Ym, Yc;
  assemble_pair32(f, m, f.Z[m], f.Z[(N - m) & (N - 1)], n <= half ? pass : 0, in, &Ym, &Yc);
  return n <= half ? Ym : Yc;
}

// Column pass: for n1 in this CTA's B columns, transform x[n1 + N1 n2] over
// n2 (length N2), multiply by exp(-+2 pi i n1 k2 / N), store to
// out[k2 N1 + n1].
// The Newton statistics of a step (iteration sum and maximum) start at zero:
// the pass-1 spectral kernels reset them (one thread per fault), and both
// Newton passes of the step run after those kernels have completed.
template <class R>
__device__ __forceinline__ void reset_newton_stats(const DevFault<R>& f, int pass, bool leader) {
  if (pass == 1 && leader && f.it_sum) {
    *f.it_sum = 0ull;
    *f.it_max = 0;
  }
}

template <class R, bool INV, int PRO>
__device__ __forceinline__ void col_body(const FftGeom& g, const Cx<R>* __restrict__ tw,
                                         const Cx<R>* __restrict__ in, Cx<R>* __restrict__ out,
                                         const DevFault<R>& f, int pass, int m_dt, double dt) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int M = g.N2, B = g.Bc;
  C* twm = buf + B * M;
  const int tid = threadIdx.x, nth = blockDim.x;
  if (PRO != PRO_LOAD) reset_newton_stats(f, pass, blockIdx.x == 0 && tid == 0);
  // the status word only changes in k_newton, never while this kernel runs
  if (PRO != PRO_LOAD && *f.status) return;
  for (int j = tid; j < (M >> 1); j += nth) twm[j] = tw[j * g.N1];
  const int c0 = blockIdx.x * B;
  for (int t = tid; t < B * M; t += nth) {
    const int b = t % B;
    const int n2 = t / B;
    const int n = c0 + b + g.N1 * n2;
    C v;
    if (PRO == PRO_LOAD) {
      v = in[n];
    } else if (PRO == PRO_PASS) {
      // predictor slip rate of this pass (Sec. 3.3): V, then (V + V1)/2; the
      // precision form has Vbar + i kappa Vbar ready in FP32 (written by the
      // commit for pass 1, by the pass-1 Newton for pass 2)
      if constexpr (sizeof(R) == 4) {
        if (f.zin1) {
          v = (pass == 1) ? f.zin1[n] : f.zin2[n];
          buf[b * M + n2] = v;
          continue;
        }
      }
      const double vb = (pass == 1) ? f.V[n] : 0.5 * (f.V[n] + f.V1[n]);
      v.x = static_cast<R>(vb);
      v.y = static_cast<R>(f.kappa[n] * vb);
    } else {
      if constexpr (sizeof(R) == 4) {
        v = f.U2f ? assemble32_at(f, n, pass, m_dt, dt) : assemble<R>(f, n, pass, m_dt, dt);
      } else {
        v = assemble<R>(f, n, pass, m_dt, dt);
      }
    }
    buf[b * M + n2] = v;
  }
  __syncthreads();
  fft_batch<C, INV>(buf, g.lgN2, B, twm, tid, nth);
  for (int t = tid; t < B * M; t += nth) {
    const int b = t % B;
    const int k2 = t / B;
    const int n1 = c0 + b;
    C w = tw[n1 * k2];
    if (INV) w.y = -w.y;
    out[k2 * g.N1 + n1] = cmul(buf[b * M + k2], w);
  }
}

template <class R, bool INV, int PRO>
__global__ void k_col(const FftGeom g, const Cx<R>* __restrict__ tw, const Cx<R>* __restrict__ in,
                      Cx<R>* __restrict__ out, const __grid_constant__ DevFault<R> f, int pass, int m_dt,
                      double dt) {
  col_body<R, INV, PRO>(g, tw, in, out, f, pass, m_dt, dt);
}

// Batched column pass: member blockIdx.y of an ensemble of equal-N faults.
template <class R, bool INV, int PRO>
__global__ void k_col_b(const FftGeom g, const DevFault<R>* __restrict__ fs, int pass, int m_dt) {
  const DevFault<R>& f = fs[blockIdx.y];
  col_body<R, INV, PRO>(g, f.tw, nullptr, f.zt, f, pass, m_dt, m_dt * f.dt_min);
}

// ------------------------------------------------ FP32 single-CTA spectral pass
// Radix-8/4/2 Stockham FFT held in registers between shared-memory stages:
// N/8 threads, each owning 8 values per stage.  Stage with sub-transform
// length Ns and radix R, for j < N/R: k = j mod Ns, v_r = A[j + r N/R]
// times exp(-+2 pi i r k / (Ns R)), an R-point DFT, and
// B[(j - k) R + k + r Ns] = V_r (self-sorting: natural order after the last
// stage).  Twiddles come from the N/2-entry table exp(-2 pi i a / N).
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// v * w8^K with w8 = exp(-sg 2 pi i / 8): sg = +1 forward, -1 inverse
// (one code path for both directions keeps the kernels small)
template <int K>
__device__ __forceinline__ float2 rot8(float2 v, float sg) {
  constexpr float c = 0.70710678118654752f;
  if constexpr (K == 0) return v;
  if constexpr (K == 1) return make_float2(c * fmaf(sg, v.y, v.x), c * fmaf(-sg, v.x, v.y));
  if constexpr (K == 2) return make_float2(sg * v.y, -sg * v.x);
  if constexpr (K == 3) return make_float2(c * fmaf(sg, v.y, -v.x), -c * fmaf(sg, v.x, v.y));
  return v;
}

template <int K>
__device__ __forceinline__ void bfly(float2& a, float2& b, float sg) {
  const float2 s = f2add(a, b), d = f2sub(a, b);
  a = s;
  b = rot8<K>(d, sg);
}

// In-place DFTs of 8, 4 and 2 points (radix-2 decimation in frequency),
// results in natural order.
__device__ __forceinline__ void dft8(float2 (&v)[8], float sg) {
  bfly<0>(v[0], v[4], sg);
  bfly<1>(v[1], v[5], sg);
  bfly<2>(v[2], v[6], sg);
  bfly<3>(v[3], v[7], sg);
  bfly<0>(v[0], v[2], sg);
  bfly<2>(v[1], v[3], sg);
  bfly<0>(v[4], v[6], sg);
  bfly<2>(v[5], v[7], sg);
  bfly<0>(v[0], v[1], sg);
  bfly<0>(v[2], v[3], sg);
  bfly<0>(v[4], v[5], sg);
  bfly<0>(v[6], v[7], sg);
  // bit reversal of 3 bits: swap 1<->4, 3<->6
  float2 t = v[1];
  v[1] = v[4];
  v[4] = t;
  t = v[3];
  v[3] = v[6];
  v[6] = t;
}

template <int O, int E>
__device__ __forceinline__ void dft4(float2 (&v)[E], float sg) {
  bfly<0>(v[O + 0], v[O + 2], sg);
  bfly<2>(v[O + 1], v[O + 3], sg);
  bfly<0>(v[O + 0], v[O + 1], sg);
  bfly<0>(v[O + 2], v[O + 3], sg);
  const float2 t = v[O + 1];
  v[O + 1] = v[O + 2];
  v[O + 2] = t;
}

// One Stockham stage over buf (length L = 2^LGL, L/EPT threads holding EPT
// values each, tid < L/EPT)
// after sub-transforms of length Ns = 2^lgNs: for j < L/R, k = j mod Ns,
// v_r = A[j + r L/R] exp(-sg 2 pi i r k / (Ns R)), an R-point DFT, and
// A[(j - k) R + k + r Ns] = V_r (self-sorting; natural order after the last
// stage).  Twiddles come from the L/2-entry table exp(-2 pi i a / L); all
// index arithmetic is shifts and masks of compile-time sizes.
template <int R, int LGL, int EPT = 8>
__device__ __forceinline__ void stockham_stage(float2* buf, const float2* tw, int lgNs, int tid, float sg) {
  constexpr int L = 1 << LGL;
  constexpr int NB = EPT / R;  // butterflies per thread
  constexpr int LGR = R == 8 ? 3 : (R == 4 ? 2 : 1);
  constexpr int nth = L / EPT;
  constexpr int stride = L / R;
  constexpr int half = L >> 1;
  const int Ns = 1 << lgNs;
  float2 v[EPT];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int j = tid + q * nth;
    const int k = j & (Ns - 1);
    const int tstep = k << (LGL - lgNs - LGR);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 x = buf[j + r * stride];
      if (r > 0) {
        const int a = r * tstep;
        float2 w = a < half ? tw[a] : make_float2(-tw[a - half].x, -tw[a - half].y);
        w.y *= sg;
        x = f2mul(x, w);
      }
      v[q * R + r] = x;
    }
  }
  if constexpr (R == 8) {
    dft8(v, sg);
  } else if constexpr (R == 4) {
    dft4<0>(v, sg);
    if constexpr (EPT == 8) dft4<4>(v, sg);
  } else {
#pragma unroll
    for (int q = 0; q < EPT / 2; ++q) bfly<0>(v[2 * q], v[2 * q + 1], sg);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int j = tid + q * nth;
    const int k = j & (Ns - 1);
    const int base = ((j - k) << LGR) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[base + r * Ns] = v[q * R + r];
  }
  __syncthreads();
}

// FFT of length 2^LGL in buf: sg = +1 forward, -1 unscaled inverse.
// EPT = 8: radix-8 stages (+4 or 2); EPT = 4: radix-4 stages (+2), twice
// the threads for the same length.
template <int LGL, int EPT = 8>
__device__ __noinline__ void fft_r8(float2* buf, const float2* tw, int tid, float sg) {
  if constexpr (EPT == 8) {
#pragma unroll 1
    for (int s = 0; s < LGL / 3; ++s) stockham_stage<8, LGL>(buf, tw, 3 * s, tid, sg);
    if constexpr (LGL % 3 == 2) stockham_stage<4, LGL>(buf, tw, 3 * (LGL / 3), tid, sg);
    if constexpr (LGL % 3 == 1) stockham_stage<2, LGL>(buf, tw, 3 * (LGL / 3), tid, sg);
  } else {
#pragma unroll 1
    for (int s = 0; s < LGL / 2; ++s) stockham_stage<4, LGL, 4>(buf, tw, 2 * s, tid, sg);
    if constexpr (LGL % 2 == 1) stockham_stage<2, LGL, 4>(buf, tw, 2 * (LGL / 2), tid, sg);
  }
}

// Whole spectral side of one pass of the precision form (FP32 FFTs) for
// N < kClusterMinN in one CTA of N/8 threads, with no FP64 arithmetic: the
// input Vbar + i kappa Vbar comes prepared in FP32 (zin1 for pass 1, written
// at commit; zin2 for pass 2, written by the pass-1 Newton), forward FFT,
// assembly of each mode pair (m, N-m) in FP32 (Sec. 3.1, Sec. 3.3 step (2)),
// inverse FFT, scaled output tau_el + i sigma_el.  Pass 2 leaves U, Q of the
// step (FP32) for the commit.  Shared memory: N complex values and N/2
// twiddles.
template <int LGN>
__device__ __forceinline__ void spectral_fused_body(const DevFault<float>& f, int pass, int m_dt, double dt) {
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int N = 1 << LGN, half = N >> 1, nth = N / 8;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw = buf + N;
  const int tid = threadIdx.x;
  __shared__ unsigned s_skip;
  pdl_trigger();
  pdl_wait();
  reset_newton_stats(f, pass, tid == 0);
  // the status word is read beside the inputs and checked once they are in
  if (tid == 0) s_skip = *f.status;
  // nth = N/8: each thread owns 4 twiddles, 8 inputs and at most 5 modes
  // (m = tid + q nth <= N/2) of the assembly; every global input is loaded
  // up front (one memory latency), into registers.
  constexpr int kMpt = 5;
  ModeIn min_[kMpt];
#pragma unroll
  for (int q = 0; q < kMpt; ++q) {
    const int m = tid + q * nth;
    if (m <= half) min_[q] = load_mode_in(f, m, m_dt, dt);
  }
  {
    const C* zin = pass == 1 ? f.zin1 : f.zin2;
    C tv[4], zv[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) tv[q] = f.tw[tid + q * nth];
#pragma unroll
    for (int q = 0; q < 8; ++q) zv[q] = zin[tid + q * nth];
#pragma unroll
    for (int q = 0; q < 4; ++q) tw[tid + q * nth] = tv[q];
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[tid + q * nth] = zv[q];
  }
  __syncthreads();
  if (s_skip) return;
  fft_r8<LGN>(buf, tw, tid, 1.0f);
#pragma unroll
  for (int q = 0; q < kMpt; ++q) {
    const int m = tid + q * nth;
    if (m <= half) {
      C Ym, Yc;
      assemble_pair32(f, m, buf[m], buf[(N - m) & (N - 1)], pass, min_[q], &Ym, &Yc);
      buf[m] = Ym;
      if (m > 0 && m < half) buf[N - m] = Yc;
    }
  }
  __syncthreads();
  fft_r8<LGN>(buf, tw, tid, -1.0f);
  const float scale = 1.0f / static_cast<float>(N);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int n = tid + q * nth;
    f.y[n] = make_float2(buf[n].x * scale, buf[n].y * scale);
  }
}

template <int LGN>
__global__ void __launch_bounds__((1 << LGN) / 8) k_spectral_fused(const __grid_constant__ DevFault<float> f,
                                                                   int pass, int m_dt, double dt) {
  spectral_fused_body<LGN>(f, pass, m_dt, dt);
}

template <int LGN>
__global__ void __launch_bounds__((1 << LGN) / 8) k_spectral_fused_b(const DevFault<float>* __restrict__ fs,
                                                                     int pass, int m_dt) {
  const DevFault<float>& f = fs[blockIdx.x];
  spectral_fused_body<LGN>(f, pass, m_dt, m_dt * f.dt_min);
}


// ------------------------------------ FP32 spectral pass on a CTA cluster
// The same pass spread over a cluster of C = cluster_ctas(N) CTAs (one SM each),
// for kClusterMinN <= N <= kFusedMaxN: four-step FFT with N = N1 N2,
// element n = n1 + N1 n2, mode m = k2 + N2 k1.  CTA c owns the columns
// n1 in [c N1/C, (c+1) N1/C) and N2/C rows k2, taken from the sequence
// 0, N2/2, 1, N2-1, 2, N2-2, ... so that a row and its mirror N2 - k2 (the
// rows of the partners N - m) sit in the same CTA.  Forward: length-N2 FFTs
// of the CTA's columns, twiddle w_N^{n1 k2}, scatter into the row owners'
// shared memory (distributed shared memory), cluster barrier, length-N1
// FFTs of the rows; assembly of each pair (m, N-m) in place; inverse: row
// FFTs, twiddle w_N^{-n1 k2}, scatter back to the column owners, barrier,
// column FFTs, output.  N/(8C) threads per CTA, 8 values each per stage.
template <int LGN, int EPT = kClusterEPT, int CC = cluster_ctas(1 << LGN)>
struct CGeom {
  static constexpr int N = 1 << LGN;
  static constexpr int lg1 = LGN / 2, lg2 = LGN - LGN / 2;
  static constexpr int N1 = 1 << lg1, N2 = 1 << lg2;
  static constexpr int C = CC;
  static constexpr int cols = N1 / C, rows = N2 / C;
  static constexpr int ept = EPT;                 // values per thread and FFT stage
  static constexpr int nth = N / (EPT * C);
};

// Index of row k2 in the pair-adjacent sequence 0, N2/2, 1, N2-1, 2, ...
__device__ __forceinline__ int row_seq(int k2, int N2) {
  if (k2 == 0) return 0;
  if (k2 == (N2 >> 1)) return 1;
  return k2 < (N2 >> 1) ? 2 * k2 : 2 * (N2 - k2) + 1;
}
__device__ __forceinline__ int seq_row(int q, int N2) {
  if (q == 0) return 0;
  if (q == 1) return N2 >> 1;
  return (q & 1) ? N2 - (q >> 1) : (q >> 1);
}
// w_N^a from the N/2-entry table (a < N), conjugated for the inverse
__device__ __forceinline__ float2 tw_full(const float2* tw, int a, int half, bool inv) {
  float2 w = a < half ? tw[a] : make_float2(-tw[a - half].x, -tw[a - half].y);
  if (inv) w.y = -w.y;
  return w;
}

__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_map(const void* p, unsigned rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
  return out;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// Transforms of length 2^LGL (2^LGL/EPT threads each) side by side in buf.
template <int LGL, int EPT>
__device__ __forceinline__ void fft_r8_batch(float2* buf, const float2* tw, int tid, float sg) {
  constexpr int per = (1 << LGL) / EPT;
  fft_r8<LGL, EPT>(buf + (tid / per) * (1 << LGL), tw, tid % per, sg);
}

template <int LGN, int EPT, int CC>
__device__ __forceinline__ void spectral_cluster_body(const DevFault<float>& f, int pass, int m_dt, double dt) {
  using G = CGeom<LGN, EPT, CC>;
  const unsigned c = cluster_rank();
  constexpr int N = G::N, half = N >> 1, nth = G::nth;
  constexpr int per = N / G::C;  // elements per CTA (EPT per thread)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* colbuf = reinterpret_cast<float2*>(smem_raw);  // [cols][N2]
  float2* rowbuf = colbuf + per;                          // [rows][N1]
  float2* s_wf = rowbuf + per;                            // forward four-step twiddle per column element
  float2* s_wi = s_wf + per;                              // inverse four-step twiddle per row element
  float2* twc = s_wi + per;                               // w_N2^j, j < N2/2
  float2* twr = twc + (G::N2 >> 1);                       // w_N1^j, j < N1/2
  ModeIn* s_min = reinterpret_cast<ModeIn*>(twr + (G::N1 >> 1));  // assembly inputs per row element
  const int tid = threadIdx.x;
  const int n1_0 = static_cast<int>(c) * G::cols;
  const int q0 = static_cast<int>(c) * G::rows;  // first sequence index of this CTA's rows
  // every CTA of the cluster runs before any remote store (arrive now, wait later)
  cluster_arrive_relaxed();
  pdl_trigger();
  {
    // every global input up front (one memory latency), staged in shared
    // memory: the pass input, the four-step twiddles of both directions, the
    // sub-table twiddles and the assembly inputs of this CTA's primary modes.
    // Launched early behind the pass-1 Newton (pass 2), it reads before
    // pdl_wait() only what no kernel of this step writes: twiddles and the
    // running and history sums of the previous commit.
    const float2* zin = pass == 1 ? f.zin1 : f.zin2;
    float2 z[EPT], wf[EPT], wi[EPT];
    ModeIn mi[EPT];
    float2 tcv = make_float2(0.f, 0.f), trv = tcv;
    if (tid < (G::N2 >> 1)) tcv = f.tw[tid * G::N1];
    if (tid < (G::N1 >> 1)) trv = f.tw[tid * G::N2];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = tid + q * nth;
      wf[q] = tw_full(f.tw, (n1_0 + e / G::N2) * (e % G::N2), half, false);
      const int k2 = seq_row(q0 + e / G::N1, G::N2);
      wi[q] = tw_full(f.tw, (e % G::N1) * k2, half, true);
      const int m = k2 + G::N2 * (e % G::N1);
      if (m <= half) mi[q] = load_mode_in(f, m, m_dt, dt);
    }
    // pass 1 is launched behind completed kernels: its input joins the loads
    // above; pass 2's input is written by the pass-1 Newton it waits for
    if (pass == 1) {
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = tid + q * nth;
        z[q] = zin[(n1_0 + e % G::cols) + G::N1 * (e / G::cols)];
      }
    }
    pdl_wait();
    reset_newton_stats(f, pass, c == 0 && tid == 0);
    if (pass != 1) {
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = tid + q * nth;
        z[q] = zin[(n1_0 + e % G::cols) + G::N1 * (e / G::cols)];
      }
    }
    if (tid < (G::N2 >> 1)) twc[tid] = tcv;
    if (tid < (G::N1 >> 1)) twr[tid] = trv;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = tid + q * nth;
      colbuf[(e % G::cols) * G::N2 + e / G::cols] = z[q];
      s_wf[e] = wf[q];
      s_wi[e] = wi[q];
      s_min[e] = mi[q];
    }
  }
  __syncthreads();
  fft_r8_batch<G::lg2, EPT>(colbuf, twc, tid, 1.0f);
  cluster_wait();
  // twiddle w_N^{n1 k2}, scatter to the row owners
#pragma unroll 1
  for (int e = tid; e < per; e += nth) {
    const int b = e / G::N2, k2 = e % G::N2;
    const int sq = row_seq(k2, G::N2);
    st_cluster(cluster_map(rowbuf + (sq % G::rows) * G::N1 + n1_0 + b, static_cast<unsigned>(sq / G::rows)),
               f2mul(colbuf[e], s_wf[e]));
  }
  cluster_arrive();
  cluster_wait();
  fft_r8_batch<G::lg1, EPT>(rowbuf, twr, tid, 1.0f);
  // assembly of the pairs (m, N-m) held by this CTA, in place
#pragma unroll 1
  for (int e = tid; e < per; e += nth) {
    const int r = e / G::N1, k1 = e % G::N1;
    const int k2 = seq_row(q0 + r, G::N2);
    const int m = k2 + G::N2 * k1;
    if (m > half) continue;
    int k2p, k1p;
    if (k2 == 0) {
      k2p = 0;
      k1p = (G::N1 - k1) & (G::N1 - 1);
    } else {
      k2p = (k2 == (G::N2 >> 1)) ? k2 : G::N2 - k2;
      k1p = G::N1 - 1 - k1;
    }
    const int ep = (row_seq(k2p, G::N2) - q0) * G::N1 + k1p;
    float2 Ym, Yc;
    assemble_pair32(f, m, rowbuf[e], rowbuf[ep], pass, s_min[e], &Ym, &Yc);
    rowbuf[e] = Ym;
    if (ep != e) rowbuf[ep] = Yc;
  }
  __syncthreads();
  fft_r8_batch<G::lg1, EPT>(rowbuf, twr, tid, -1.0f);
  // twiddle w_N^{-n1 k2}, scatter back to the column owners
#pragma unroll 1
  for (int e = tid; e < per; e += nth) {
    const int r = e / G::N1, n1 = e % G::N1;
    const int k2 = seq_row(q0 + r, G::N2);
    st_cluster(cluster_map(colbuf + (n1 % G::cols) * G::N2 + k2, static_cast<unsigned>(n1 / G::cols)),
               f2mul(rowbuf[e], s_wi[e]));
  }
  cluster_arrive();
  cluster_wait();
  fft_r8_batch<G::lg2, EPT>(colbuf, twc, tid, -1.0f);
  const float scale = 1.0f / static_cast<float>(N);
#pragma unroll 1
  for (int e = tid; e < per; e += nth) {
    const float2 v = colbuf[(e % G::cols) * G::N2 + e / G::cols];
    f.y[(n1_0 + e % G::cols) + G::N1 * (e / G::cols)] = make_float2(v.x * scale, v.y * scale);
  }
}

template <int LGN, int EPT>
__global__ void __launch_bounds__(CGeom<LGN, EPT>::nth) k_spectral_cluster(const __grid_constant__ DevFault<float> f,
                                                                            int pass, int m_dt, double dt) {
  spectral_cluster_body<LGN, EPT, cluster_ctas(1 << LGN)>(f, pass, m_dt, dt);
}

template <int LGN, int EPT>
__global__ void __launch_bounds__(CGeom<LGN, EPT, batch_cluster_ctas(1 << LGN)>::nth)
    k_spectral_cluster_b(const DevFault<float>* __restrict__ fs, int pass, int m_dt) {
  constexpr int CC = batch_cluster_ctas(1 << LGN);
  const DevFault<float>& f = fs[blockIdx.x / CC];
  spectral_cluster_body<LGN, EPT, CC>(f, pass, m_dt, m_dt * f.dt_min);
}

// Row pass: for k2 in this CTA's B rows, transform t[k2 N1 + n1] over n1
// (length N1) and store to out[k2 + N2 k1], times scale.
template <class R, bool INV>
__device__ __forceinline__ void row_body(const FftGeom& g, const Cx<R>* __restrict__ tw,
                                         const Cx<R>* __restrict__ in, Cx<R>* __restrict__ out, R scale,
                                         const unsigned* status) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int M = g.N1, B = g.Br;
  C* twm = buf + B * M;
  const int tid = threadIdx.x, nth = blockDim.x;
  if (status && *status) return;
  for (int j = tid; j < (M >> 1); j += nth) twm[j] = tw[j * g.N2];
  const int c0 = blockIdx.x * B;
  for (int t = tid; t < B * M; t += nth) {
    const int n1 = t % M;
    const int b = t / M;
    buf[b * M + n1] = in[(c0 + b) * g.N1 + n1];
  }
  __syncthreads();
  fft_batch<C, INV>(buf, g.lgN1, B, twm, tid, nth);
  for (int t = tid; t < B * M; t += nth) {
    const int b = t % B;
    const int k1 = t / B;
    C v = buf[b * M + k1];
    v.x *= scale;
    v.y *= scale;
    out[(c0 + b) + g.N2 * k1] = v;
  }
}

template <class R, bool INV>
__global__ void k_row(const FftGeom g, const Cx<R>* __restrict__ tw, const Cx<R>* __restrict__ in,
                      Cx<R>* __restrict__ out, R scale, const unsigned* status) {
  row_body<R, INV>(g, tw, in, out, scale, status);
}

template <class R, bool INV>
__global__ void k_row_b(const FftGeom g, const DevFault<R>* __restrict__ fs) {
  const DevFault<R>& f = fs[blockIdx.y];
  row_body<R, INV>(g, f.tw, f.zt, INV ? f.y : f.Z, INV ? R(1.0 / g.N) : R(1), f.status);
}

// ---------------------------------------------------- history convolution
// Ring slot i of mode n (i = 0 newest) holds the spectra of the interval
// lying i dt_min before the current step; with a step of m dt_min it meets
// the weight of interval j = i + m (Sec. 3.3, midpoint weights of Sec. 3.3).
template <class R> struct Acc4 { R tr, ti, nr, ni; };

__device__ __forceinline__ void slot_fma(Acc4<double>& a, const Slot64& s, const double2 w) {
  a.tr = fma(w.x, s.t.x, a.tr);
  a.ti = fma(w.x, s.t.y, a.ti);
  a.nr = fma(w.y, s.n.x, a.nr);
  a.ni = fma(w.y, s.n.y, a.ni);
}
__device__ __forceinline__ void slot_fma(Acc4<float>& a, const float4& s, const float2 w) {
  a.tr = fmaf(w.x, s.x, a.tr);
  a.ti = fmaf(w.x, s.y, a.ti);
  a.nr = fmaf(w.y, s.z, a.nr);
  a.ni = fmaf(w.y, s.w, a.ni);
}
__device__ __forceinline__ Slot64 ld_slot(const Slot64* p) {
  Slot64 s;
  s.t = __ldg(&p->t);
  s.n = __ldg(&p->n);
  return s;
}
__device__ __forceinline__ float4 ld_slot(const float4* p) { return __ldg(p); }

template <class R> struct HistCfg;
template <> struct HistCfg<double> { static constexpr int kUnroll = 4; };
template <> struct HistCfg<float> { static constexpr int kUnroll = 8; };

constexpr int kHistThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per chunk of consecutive slots of one mode: lanes stride over the
// slots (each warp load is one contiguous segment), reduce with shuffles.  A
// mode split over several chunks is finished by the warp whose chunk
// completes last (atomic counter per mode, no waiting): it adds the partial
// sums in chunk order, so the result does not depend on scheduling.
// BATCH: the chunks of an ensemble, chunk.member selects the fault in fs
// (partial sums, counters and the work counter of fs[*] are the ensemble's).
template <class R, bool BATCH>
__global__ void __launch_bounds__(kHistThreads)
    k_history_t(const __grid_constant__ DevFault<R> f0, const DevFault<R>* __restrict__ fs,
                const Chunk* __restrict__ chunks, int nchunks, int* work, int m_dt) {
  if (!BATCH && *f0.status) return;  // the status word does not change while this kernel runs
  constexpr int U = HistCfg<R>::kUnroll;
  const int lane = threadIdx.x & 31;
  // chunks are handed out dynamically (counter zeroed before the launch)
  int c = 0;
  if (lane == 0) c = atomicAdd(work, 1);
  c = __shfl_sync(0xffffffffu, c, 0);
  for (; c < nchunks; c = __shfl_sync(0xffffffffu, c, 0)) {
    const Chunk cd = chunks[c];
    const DevFault<R>& f = BATCH ? fs[cd.pad] : f0;
    if (BATCH && *f.status) {
      if (lane == 0) c = atomicAdd(work, 1);
      continue;
    }
    const int n = cd.mode;
    const int Rn = f.Rn[n];
    const int h = f.head[n];
    const int64_t iend = min(cd.i1, static_cast<int64_t>(f.Mn[n]) - m_dt);
    const Slot<R>* ring = f.ring + f.ring_off[n];
    const W2<R>* w = f.w + f.w_off[n] + m_dt;
    Acc4<R> acc = {R(0), R(0), R(0), R(0)};
    for (int64_t i = cd.i0 + lane; i < iend; i += 32 * U) {
      Slot<R> sv[U];
      W2<R> wv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t ii = i + 32 * u;
        if (ii < iend) {
          int64_t slot = h + ii;
          if (slot >= Rn) slot -= Rn;
          sv[u] = ld_slot(ring + slot);
          wv[u] = __ldg(w + ii);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (i + 32 * u < iend) slot_fma(acc, sv[u], wv[u]);
    }
    // reduce in the accumulation precision (FP32 partial sums in the precision
    // form), widen once per chunk for the cross-chunk sum
    const double4 v = make_double4(static_cast<double>(warp_sum(acc.tr)), static_cast<double>(warp_sum(acc.ti)),
                                   static_cast<double>(warp_sum(acc.nr)), static_cast<double>(warp_sum(acc.ni)));
    const int cur = c;
    if (lane == 0) c = atomicAdd(work, 1);
    if (cd.count == 1) {
      if (lane == 0) {
        f.AT[n] = make_double2(v.x, v.y);
        f.AN[n] = make_double2(v.z, v.w);
        if (f.AT32) {
          f.AT32[n] = make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
          f.AN32[n] = make_float2(static_cast<float>(v.z), static_cast<float>(v.w));
        }
      }
      continue;
    }
    int prev = 0;
    if (lane == 0) {
      f.partial[cur] = v;
      __threadfence();
      prev = atomicAdd(f.counter + n, 1);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev == cd.count - 1) {
      __threadfence();
      double4 r = make_double4(0.0, 0.0, 0.0, 0.0);
      for (int q = lane; q < cd.count; q += 32) {
        const double2* pp = reinterpret_cast<const double2*>(f.partial + cd.first + q);
        const double2 p0 = __ldcg(pp), p1 = __ldcg(pp + 1);
        r.x += p0.x;
        r.y += p0.y;
        r.z += p1.x;
        r.w += p1.y;
      }
      r = make_double4(warp_sum(r.x), warp_sum(r.y), warp_sum(r.z), warp_sum(r.w));
      if (lane == 0) {
        f.AT[n] = make_double2(r.x, r.y);
        f.AN[n] = make_double2(r.z, r.w);
        if (f.AT32) {
          f.AT32[n] = make_float2(static_cast<float>(r.x), static_cast<float>(r.y));
          f.AN32[n] = make_float2(static_cast<float>(r.z), static_cast<float>(r.w));
        }
        f.counter[n] = 0;
      }
    }
  }
}

// ---------------------------------------------- history sweep (bulk-async)
// The history convolution of a single fault as a stream through shared
// memory: each CTA takes a contiguous range of chunks (at most kSweepSlots
// lags of one mode each); one thread issues cp.async.bulk copies of the
// chunk's ring slots (one or two pieces, the ring wraps) and weights into a
// kSweepStages-deep ring of stage buffers, completion tracked by an mbarrier
// per stage; all threads reduce the stage and the CTA writes one partial sum
// per chunk (no atomics).  A chunk's sum runs over its lags in a fixed
// order, so results do not depend on scheduling.  Every wait is bounded: on
// a timeout the kernel sets SBIEM_FLAG_WAIT, waits (bounded) for its copies
// in flight and returns.
// Shapes of the sweep: lags per chunk (= stage buffer) x stages in flight per
// CTA.  Shape 0: 512 x 4 (FP32, 12 KB stages) / 256 x 4 (FP64, 12 KB);
// shape 1: twice the lags; shape 2: twice the stages; shape 3: 4x the lags, 2
// stages; shape 4: shape 3's chunks in one stage (49 KB), for the sweep that
// runs beside the spectral passes: two of its CTAs and a pass CTA share an SM.
template <class R, int SH> struct SweepCfg {
  static constexpr int kBase = sizeof(R) == 4 ? 512 : 256;
  static constexpr int kSlots = SH == 1 ? 2 * kBase : (SH >= 3 ? 4 * kBase : kBase);
  static constexpr int kStages = SH == 2 ? 8 : (SH == 3 ? 2 : (SH == 4 ? 1 : 4));
};
constexpr int kSweepShapes = 5;
constexpr int kSweepThreads = 128;
// Threads of a sweep CTA: the on-chip weight form evaluates a polynomial per
// lag and needs twice the warps to hide its latency.
__host__ __device__ constexpr int sweep_threads(bool gen) { return gen ? 2 * kSweepThreads : kSweepThreads; }
constexpr long long kSpinLimit = SBIEM_WAIT_LIMIT_DEFAULT;  // try_wait polls before a wait is declared stuck

// A stage holds a chunk's ring slots and its weight run (left unused by a
// chunk whose weights are evaluated on chip).
template <class R, int SH>
__host__ __device__ constexpr size_t sweep_stage_bytes() {
  return static_cast<size_t>(SweepCfg<R, SH>::kSlots) * sizeof(Slot<R>) +
         static_cast<size_t>(SweepCfg<R, SH>::kSlots + 2) * sizeof(W2<R>);
}

// On-chip weights: kGenDeg + 1 coefficient pairs (T, N) per piece of width
// kGenH, kGenF4 float4 per piece, read through L1 (the table is a few tens
// of KB; a thread loads one piece per block of lags).
constexpr int kGenPairs = kGenDeg + 1;
constexpr int kGenF4 = kGenPairs / 2;
static_assert(kGenPairs % 2 == 0, "coefficient pairs come two per float4");
constexpr float kGenHf = static_cast<float>(kGenH);
constexpr float kGenInvH = static_cast<float>(1.0 / kGenH);

// Two FP32 fused multiply-adds in one packed instruction (fma.rn.f32x2):
// each lane rounds exactly as fmaf does.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ra, rb, rc, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

// The weights of a thread's block of kGenBlock consecutive lags come from
// one piece: the block starts at lag j (s0 = (j + 1/2) ds, ds = dsh + dsl as
// two floats) in piece q; s0 jf dsh is rounded once and its error comes
// exactly from an FMA, so the offset within the piece (q kGenH exact,
// p - q kGenH exact by Sterbenz) carries s to about 1e-8 absolute.  The
// piece's polynomial holds over kGenSpan piece widths, so the block stays on
// it while (kGenBlock - 1) ds <= (kGenSpan - 1) kGenH: modes with ds up to
// kGenDsBlockMax.
// Modes with ds above that and up to kGenDsBlock4Max take blocks of four
// lags (two per thread and stage).
constexpr int kGenBlock = 8;
constexpr int kGenBlock4 = 4;
constexpr float kGenTScale = static_cast<float>(2.0 / (kGenSpan * kGenH));  // dt / ds
static_assert((kGenBlock - 1) * kGenDsBlockMax <= (kGenSpan - 1.0) * kGenH, "blocks stay on their piece");
static_assert((kGenBlock4 - 1) * kGenDsBlock4Max <= (kGenSpan - 1.0) * kGenH, "blocks stay on their piece");
static_assert(sweep_threads(true) * kGenBlock == SweepCfg<float, 3>::kSlots, "a GEN stage is one block per thread");

// (w^T, w^N) = the piece's polynomial at t: Horner on the coefficient pairs
// (c[i].x, c[i].y) = pair 2i, (c[i].z, c[i].w) = pair 2i + 1, two lanes per
// packed FMA.
__device__ __forceinline__ float2 gen_horner(const float4 (&c)[kGenF4], float t) {
  const float2 tt = make_float2(t, t);
  float2 w = make_float2(c[kGenF4 - 1].z, c[kGenF4 - 1].w);
#pragma unroll
  for (int i = kGenF4 - 1; i >= 0; --i) {
    if (i < kGenF4 - 1) w = ffma2(w, tt, make_float2(c[i].z, c[i].w));
    w = ffma2(w, tt, make_float2(c[i].x, c[i].y));
  }
  return w;
}

// acc += (wT (s.x, s.y), wN (s.z, s.w)) in two packed FMAs.
__device__ __forceinline__ void slot_fma2(float2& at, float2& an, const float4& s, const float2 w) {
  at = ffma2(make_float2(w.x, w.x), make_float2(s.x, s.y), at);
  an = ffma2(make_float2(w.y, w.y), make_float2(s.z, s.w), an);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of bar: at most `limit` polls; false when
// the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit = kSpinLimit) {
  for (long long k = 0; k < limit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The same copy with an L2 eviction policy (createpolicy): the ensemble
// sweep marks its ring slots evict-first so that the weight runs its
// members share stay in L2.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                              uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// s + c += a with the rounding error of the addition carried in c (Knuth's
// TwoSum; FP32 only -- an FP64 sum needs no compensation here).
__device__ __forceinline__ void two_sum_add(float& s, float& c, float a) {
  const float t = s + a;
  const float bb = t - s;
  c += (s - (t - bb)) + (a - bb);
  s = t;
}
__device__ __forceinline__ void two_sum_add(double& s, double& /*c*/, double a) { s += a; }

// Fixed-order tree sum of a warp's values, valid in lane 0.  Only the lanes
// that keep a partial sum add (lane < o), so the FP64 pipe (scarce on GB300)
// does 31 additions per value instead of 160.
template <class T>
__device__ __forceinline__ T warp_reduce_to_lane0(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T u = __shfl_down_sync(0xffffffffu, v, o);
    if (lane < o) v += u;
  }
  return v;
}

// Copy plan of one chunk (computed ahead by all threads, read by the
// issuing thread): up to two ring pieces and one 16-byte aligned weight run.
struct SweepPlan {
  const void* r1;
  const void* r2;
  const void* wsrc;
  unsigned b1, b2, bw;
  int len, par, mode, member;
  // on-chip weights (gen != 0): weight index of the chunk's first slot, the
  // mode's ds as two floats and the two fields' windows
  int gen, j0, mt, mn;
  float dsh, dsl;
};
constexpr int kPlanRing = 64;  // plans held in shared memory (a ring by chunk index)

// On-chip weights of B consecutive lags [base, base + B) of a stage (B a
// power of two, base < L): one piece of the table serves the block, the
// lags are read in an order rotated by the lane (so the lanes of a quarter
// warp hit different bank groups), and (at, an) accumulate the products.
template <int B>
__device__ __forceinline__ void gen_block(const SweepPlan& pk, const float4* __restrict__ sring, int base, int L,
                                          int lane, const float4* __restrict__ wtab, int wtab_pieces, float2& at,
                                          float2& an) {
  const float jf = static_cast<float>(pk.j0 + base) + 0.5f;  // exact: lags stay below 2^23
  const float p = jf * pk.dsh;
  const float e = fmaf(jf, pk.dsl, fmaf(jf, pk.dsh, -p));
  const float qf = fminf(floorf(p * kGenInvH), static_cast<float>(wtab_pieces - 1));
  const int q = static_cast<int>(qf);
  const float t0 = fmaf(fmaf(-qf, kGenHf, p) + e, kGenTScale, -1.0f);
  const float dtv = pk.dsh * kGenTScale;
  float4 cf[kGenF4];
#pragma unroll
  for (int i = 0; i < kGenF4; ++i) cf[i] = __ldg(wtab + kGenF4 * q + i);
  const float4* blk = sring + base;
  if (base + B <= L && pk.j0 + base + B <= min(pk.mt, pk.mn)) {
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int r = (k + lane) & (B - 1);  // the lane-rotated lag order
      slot_fma2(at, an, blk[r], gen_horner(cf, fmaf(static_cast<float>(r), dtv, t0)));
    }
  } else {
    // the chunk's tail, or a field's window ending inside the block
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int r = (k + lane) & (B - 1);
      float2 w = gen_horner(cf, fmaf(static_cast<float>(r), dtv, t0));
      if (pk.j0 + base + r >= pk.mt) w.x = 0.0f;
      if (pk.j0 + base + r >= pk.mn) w.y = 0.0f;
      if (base + r < L) slot_fma2(at, an, blk[r], w);
    }
  }
}

// Chunk c of the sweep: the fault's own chunk table, or an ensemble table
// whose chunks name their member (Chunk::pad) in fs.
// gen_ds_max (GEN only): modes whose s step ds = c_s k_n dt_min is at most
// this evaluate their weights on chip, the others stream them.
template <class R, bool BATCH, bool GEN = false>
__device__ __forceinline__ SweepPlan sweep_plan(const DevFault<R>& f0, const DevFault<R>* fs, const Chunk* chunks,
                                                int c, int m_dt, float gen_ds_max = 0.0f) {
  SweepPlan pl{};
  const Chunk cd = chunks[c];
  const DevFault<R>& f = BATCH ? fs[cd.pad] : f0;
  pl.member = BATCH ? cd.pad : 0;
  const int n = cd.mode;
  const int Rn = f.Rn[n];
  const int64_t iend = min(cd.i1, static_cast<int64_t>(f.Mn[n]) - m_dt);
  const int L = iend > cd.i0 ? static_cast<int>(iend - cd.i0) : 0;
  pl.len = L;
  pl.mode = n;
  if (L == 0) return pl;
  int64_t p0 = f.head[n] + cd.i0;
  if (p0 >= Rn) p0 -= Rn;
  const int L1 = static_cast<int>(min(static_cast<int64_t>(L), Rn - p0));
  const int L2 = L - L1;
  // weights: 16-byte aligned start (two FP32 pairs per 16 bytes)
  const int64_t ws = f.w_off[n] + m_dt + cd.i0;
  constexpr int per16 = 16 / static_cast<int>(sizeof(W2<R>));  // 2 (FP32) or 1 (FP64)
  const int64_t wa = ws / per16 * per16;
  pl.par = static_cast<int>(ws - wa);
  const int wc = (pl.par + L + per16 - 1) / per16 * per16;
  const Slot<R>* ring = f.ring + f.ring_off[n];
  pl.r1 = ring + p0;
  pl.b1 = static_cast<unsigned>(L1 * sizeof(Slot<R>));
  pl.r2 = ring;
  pl.b2 = static_cast<unsigned>(L2 * sizeof(Slot<R>));
  pl.gen = 0;
  if constexpr (GEN) {
    const float4 gi = f.wgen[n];
    if (gi.x <= gen_ds_max) {
      // eight-lag blocks up to kGenDsBlockMax, four-lag blocks above
      pl.gen = gi.x <= static_cast<float>(kGenDsBlockMax) ? 1 : 2;
      pl.j0 = static_cast<int>(m_dt + cd.i0);
      pl.dsh = gi.x;
      pl.dsl = gi.y;
      pl.mt = __float_as_int(gi.z);
      pl.mn = __float_as_int(gi.w);
      pl.wsrc = nullptr;
      pl.bw = 0;
      return pl;
    }
  }
  pl.wsrc = f.w + wa;
  pl.bw = static_cast<unsigned>(wc * sizeof(W2<R>));
  return pl;
}

// Thread 0: start the copies of a planned chunk into a stage (ring_pol != 0:
// the ring pieces under that L2 policy).
template <class R, int S>
__device__ __forceinline__ void sweep_issue(const SweepPlan& pl, unsigned char* stage_buf, uint64_t* bar,
                                            uint64_t ring_pol) {
  if (pl.len == 0) {
    mbar_arrive(bar);
    return;
  }
  unsigned char* sw = stage_buf + static_cast<size_t>(S) * sizeof(Slot<R>);
  mbar_expect_tx(bar, pl.b1 + pl.b2 + pl.bw);
  if (ring_pol) {
    bulk_g2s_hint(stage_buf, pl.r1, pl.b1, bar, ring_pol);
    if (pl.b2) bulk_g2s_hint(stage_buf + pl.b1, pl.r2, pl.b2, bar, ring_pol);
  } else {
    bulk_g2s(stage_buf, pl.r1, pl.b1, bar);
    if (pl.b2) bulk_g2s(stage_buf + pl.b1, pl.r2, pl.b2, bar);
  }
  if (pl.bw) bulk_g2s(sw, pl.wsrc, pl.bw, bar);
}

// BATCH: the chunks of an ensemble (member in Chunk::pad), descriptors in fs;
// members whose step failed are swept anyway (their sums are not written).
// GEN (FP32): chunks of modes with ds <= gen_ds_max evaluate their weights
// from the piecewise-polynomial table wtab (wtab_pieces pieces, global,
// read through L1) instead of copying them with the ring slots.
// The sweep of one CTA over its chunks [c0, c0 + nk) (nk >= 1).  Returns
// false when a copy wait gave up; *k_stop is then the first chunk (counted
// from c0) whose sum was not written, and every copy in flight has landed.
template <class R, int SH, bool BATCH, bool GEN>
__device__ __forceinline__ bool sweep_chunks(const DevFault<R>& f, const DevFault<R>* __restrict__ fs,
                                             const Chunk* __restrict__ chunks, int c0, int nk,
                                             double4* __restrict__ partial, int m_dt,
                                             const float4* __restrict__ wtab, int wtab_pieces, float gen_ds_max,
                                             long long lim, bool skip_on_status, int* k_stop,
                                             bool ring_evict_first = false) {
  static_assert(!GEN || sizeof(R) == 4, "on-chip weights belong to the FP32 form");
  constexpr int S = SweepCfg<R, SH>::kSlots;
  constexpr int kSweepStages = SweepCfg<R, SH>::kStages;
  constexpr size_t SB = sweep_stage_bytes<R, SH>();
  constexpr int NT = sweep_threads(GEN);
  constexpr int NW = NT / 32;
  extern __shared__ __align__(128) unsigned char sweep_smem[];
  __shared__ __align__(8) uint64_t bars[kSweepStages];
  __shared__ SweepPlan plan[kPlanRing];
  __shared__ Acc4<R> red[2][NW];
  __shared__ unsigned s_skip;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint64_t ring_pol = ring_evict_first && tid == 0 ? l2_policy_evict_first() : 0;
  *k_stop = nk;
  // one read of the status word (a concurrent pass may set it), taken beside
  // the loads of the first plans and checked once they are in: a uniform
  // exit without a memory round trip of its own before the first copy
  if (tid == 0) {
    s_skip = skip_on_status ? *f.status : 0u;
    for (int s = 0; s < kSweepStages; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // plans of the first kPlanRing chunks (one per thread)
  for (int j = tid; j < kPlanRing && j < nk; j += NT)
    plan[j] = sweep_plan<R, BATCH, GEN>(f, fs, chunks, c0 + j, m_dt, gen_ds_max);
  __syncthreads();
  if (s_skip) return true;
  if (tid == 0)
    for (int k = 0; k < kSweepStages && k < nk; ++k)
      sweep_issue<R, S>(plan[k], sweep_smem + k * SB, &bars[k], ring_pol);
  // the consumer waits take the caller's limit (sbiem_set_wait_limit); the
  // drain below always waits at the full limit, so no copy is left in flight
  // each thread accumulates a chunk in R and folds it into a compensated sum
  // over the consecutive chunks of one mode (a run may hold hundreds of
  // chunks: one plain FP32 sum of its thousands of products lost 5e-6); the
  // CTA reduces at the end of the mode's run (a segment) and writes the sum
  // at the segment's last chunk, zeros at the others
  bool stuck = false;
  int k = 0;
  Acc4<R> run = {R(0), R(0), R(0), R(0)}, cmp = {R(0), R(0), R(0), R(0)};

  for (; k < nk; ++k) {
    const int s = k % kSweepStages;
    // every kPlanRing/2 chunks: plans of the half-ring ahead (chunks
    // k + kPlanRing/2 .. k + kPlanRing - 1 replace chunks already issued)
    if (k > 0 && k % (kPlanRing / 2) == 0) {
      const int j = k + kPlanRing / 2 + tid;
      if (tid < kPlanRing / 2 && j < nk)
        plan[j % kPlanRing] = sweep_plan<R, BATCH, GEN>(f, fs, chunks, c0 + j, m_dt, gen_ds_max);
    }
    const unsigned parity = static_cast<unsigned>(k / kSweepStages) & 1u;
    const bool ok = mbar_wait(&bars[s], parity, lim);
    Acc4<R> acc = {R(0), R(0), R(0), R(0)};
    if (ok) {
      const SweepPlan& pk = plan[k % kPlanRing];
      const int L = pk.len;
      const Slot<R>* sring = reinterpret_cast<const Slot<R>*>(sweep_smem + s * SB);
      auto streamed = [&] {
        const int par = pk.par;
        const W2<R>* sw =
            reinterpret_cast<const W2<R>*>(sweep_smem + s * SB + static_cast<size_t>(S) * sizeof(Slot<R>));
#pragma unroll 4
        for (int i = tid; i < L; i += NT) slot_fma(acc, sring[i], sw[par + i]);
      };
      if constexpr (GEN) {
       if (!pk.gen) {
        streamed();
       } else {
        float2 at = make_float2(0.f, 0.f), an = make_float2(0.f, 0.f);
        if (pk.gen == 1) {
          // thread tid: lags [kGenBlock tid, kGenBlock (tid + 1)) of the chunk
          const int base = kGenBlock * tid;
          if (base < L) gen_block<kGenBlock>(pk, sring, base, L, lane, wtab, wtab_pieces, at, an);
        } else {
          // two blocks of four: lags [4 tid, 4 tid + 4) and the same half a stage on
#pragma unroll
          for (int hb = 0; hb < kGenBlock / kGenBlock4; ++hb) {
            const int base = kGenBlock4 * tid + hb * (kGenBlock4 * NT);
            if (base < L) gen_block<kGenBlock4>(pk, sring, base, L, lane, wtab, wtab_pieces, at, an);
          }
        }
        acc.tr = at.x;
        acc.ti = at.y;
        acc.nr = an.x;
        acc.ni = an.y;
       }
      } else {
        streamed();
      }
    }
    two_sum_add(run.tr, cmp.tr, acc.tr);
    two_sum_add(run.ti, cmp.ti, acc.ti);
    two_sum_add(run.nr, cmp.nr, acc.nr);
    two_sum_add(run.ni, cmp.ni, acc.ni);
    const SweepPlan &pc = plan[k % kPlanRing], &pn = plan[(k + 1) % kPlanRing];
    const bool seg_end = k + 1 == nk || pn.mode != pc.mode || pn.member != pc.member;
    if (seg_end) {
      Acc4<R> w4;
      w4.tr = warp_reduce_to_lane0(run.tr + cmp.tr);
      w4.ti = warp_reduce_to_lane0(run.ti + cmp.ti);
      w4.nr = warp_reduce_to_lane0(run.nr + cmp.nr);
      w4.ni = warp_reduce_to_lane0(run.ni + cmp.ni);
      if (lane == 0) red[k & 1][wid] = w4;
      run = {R(0), R(0), R(0), R(0)};
      cmp = {R(0), R(0), R(0), R(0)};
    }
    stuck = __syncthreads_or(!ok);
    if (stuck) break;
    if (tid == 0) {
      // the stage was read by every thread (barrier above): refill it first
      if (k + kSweepStages < nk)
        sweep_issue<R, S>(plan[(k + kSweepStages) % kPlanRing], sweep_smem + s * SB, &bars[s], ring_pol);
      double4 out = make_double4(0.0, 0.0, 0.0, 0.0);
      if (seg_end) {
        Acc4<R> t = red[k & 1][0];
#pragma unroll
        for (int w = 1; w < NW; ++w) {
          const Acc4<R> u = red[k & 1][w];
          t.tr += u.tr;
          t.ti += u.ti;
          t.nr += u.nr;
          t.ni += u.ni;
        }
        out = make_double4(static_cast<double>(t.tr), static_cast<double>(t.ti), static_cast<double>(t.nr),
                           static_cast<double>(t.ni));
      }
      partial[c0 + k] = out;
    }
  }
  if (stuck && tid == 0) {
    atomicOr(BATCH ? fs[plan[k % kPlanRing].member].status : f.status, SBIEM_FLAG_WAIT);
    // copies still in flight land in this CTA's shared memory: wait for them
    // (bounded) before the CTA exits
    for (int q = k; q < nk && q < k + kSweepStages; ++q)
      mbar_wait(&bars[q % kSweepStages], static_cast<unsigned>(q / kSweepStages) & 1u);
  }
  *k_stop = k;
  return !stuck;
}

template <class R, int SH, bool BATCH, bool GEN>
__global__ void __launch_bounds__(sweep_threads(GEN), GEN ? 4 : 1)
    k_sweep(const __grid_constant__ DevFault<R> f, const DevFault<R>* __restrict__ fs,
            const Chunk* __restrict__ chunks, int nch, double4* __restrict__ partial, int m_dt,
            const float4* __restrict__ wtab, int wtab_pieces, float gen_ds_max, bool ring_evict_first) {
  // the per-mode finish may be resident already, waiting for this grid
  pdl_trigger();
  const int c0 = static_cast<int>(static_cast<int64_t>(blockIdx.x) * nch / gridDim.x);
  const int c1 = static_cast<int>(static_cast<int64_t>(blockIdx.x + 1) * nch / gridDim.x);
  if (c1 <= c0) return;
  int k_stop;
  sweep_chunks<R, SH, BATCH, GEN>(f, fs, chunks, c0, c1 - c0, partial, m_dt, wtab, wtab_pieces, gen_ds_max,
                                  BATCH ? kSpinLimit : f.spin_limit, !BATCH, &k_stop, ring_evict_first);
}

// Per-mode sums of the sweep's segment partials, one thread per mode.  The
// sweep (grid G, CTA b taking chunks [c0(b), c0(b+1)), c0(b) = b nch / G)
// leaves a mode's sum over one CTA at the CTA's last chunk of that mode and
// zeros at its other chunks, so only those chunks are read: for every CTA
// overlapping the mode's chunks [F, E), chunk min(c0(b+1), E) - 1, added in
// chunk order.  Writes (AT, AN) or, for the overlapped form, (BT, BN); the
// FP32 copies when `f32` is set.
template <class R>
__global__ void k_sweep_finish(const __grid_constant__ DevFault<R> f, double2* outT, double2* outN, bool f32,
                               int G) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  // launched early behind the sweep: its partials are read after the wait
  pdl_wait();
  if (n >= f.nmodes || *f.status) return;
  const int64_t nch = f.nchunks;
  const int64_t F = f.mfirst[n], E = F + f.mcount[n];
  double4 t = make_double4(0.0, 0.0, 0.0, 0.0);
  if (E > F) {
    auto c0 = [&](int64_t b) { return b * nch / G; };
    // the CTA holding chunk F: the largest b with c0(b) <= F
    for (int64_t b = ((F + 1) * G + nch - 1) / nch - 1; b < G && c0(b) < E; ++b) {
      const int64_t end = min(c0(b + 1), E) - 1;
      const double4 u = f.partial[end];
      t.x += u.x;
      t.y += u.y;
      t.z += u.z;
      t.w += u.w;
    }
  }
  outT[n] = make_double2(t.x, t.y);
  outN[n] = make_double2(t.z, t.w);
  if (f32 && f.AT32) {
    f.AT32[n] = make_float2(static_cast<float>(t.x), static_cast<float>(t.y));
    f.AN32[n] = make_float2(static_cast<float>(t.z), static_cast<float>(t.w));
  }
}

// Ensemble form of k_sweep_finish: one thread per (member, mode) pair
// mm[t], whose chunks are [fc[t].x, fc[t].x + fc[t].y) of the ensemble's
// chunk table.  Members whose step failed are left alone.
template <class R>
__device__ __forceinline__ void finish_pair(const DevFault<R>* __restrict__ fs, const int2* __restrict__ mm, int t,
                                            const int2* __restrict__ fc, int nch, int G,
                                            const double4* __restrict__ partial, bool ahead) {
  const int2 rn = mm[t];
  const DevFault<R>& f = fs[rn.x];
  if (*f.status) return;
  const int n = rn.y;
  const int2 q = fc[t];
  const int64_t F = q.x, E = F + q.y;
  double4 acc = make_double4(0.0, 0.0, 0.0, 0.0);
  if (E > F) {
    auto c0 = [&](int64_t b) { return b * nch / G; };
    for (int64_t b = ((F + 1) * G + nch - 1) / nch - 1; b < G && c0(b) < E; ++b) {
      // L2 reads: the partials come from other CTAs of the same grid in the persistent form
      const double2* pp = reinterpret_cast<const double2*>(partial + (min(c0(b + 1), E) - 1));
      const double2 lo = __ldcg(pp), hi = __ldcg(pp + 1);
      const double4 u = make_double4(lo.x, lo.y, hi.x, hi.y);
      acc.x += u.x;
      acc.y += u.y;
      acc.z += u.z;
      acc.w += u.w;
    }
  }
  if (ahead) {
    // overlapped form: the next step's sums without its newest interval
    f.BT[n] = make_double2(acc.x, acc.y);
    f.BN[n] = make_double2(acc.z, acc.w);
    return;
  }
  f.AT[n] = make_double2(acc.x, acc.y);
  f.AN[n] = make_double2(acc.z, acc.w);
  if (f.AT32) {
    f.AT32[n] = make_float2(static_cast<float>(acc.x), static_cast<float>(acc.y));
    f.AN32[n] = make_float2(static_cast<float>(acc.z), static_cast<float>(acc.w));
  }
}

template <class R>
__global__ void k_sweep_finish_b(const DevFault<R>* __restrict__ fs, const int2* __restrict__ mm, int TM,
                                 const int2* __restrict__ fc, int nch, int G,
                                 const double4* __restrict__ partial, bool ahead) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < TM) finish_pair<R>(fs, mm, t, fc, nch, G, partial, ahead);
}

// The ensemble's history convolution in one persistent launch (cooperative:
// every CTA is resident): each CTA sweeps its range of the members' chunk
// tables laid end to end (its (member, mode-run) sums into the partials),
// all CTAs meet at a grid barrier, then the grid adds every (member, mode)
// pair's partials.  The barrier is a counter and an epoch in device memory:
// the last CTA to arrive resets the counter and advances the epoch; the
// others poll the epoch at most bar_limit times.  A CTA that gives up sets
// SBIEM_FLAG_WAIT on every member and leaves (their steps are rejected,
// nothing is committed); a CTA whose copy wait gave up flags the members of
// the chunks it did not sum and still arrives.
struct SweepBarrier {
  unsigned* count;
  unsigned* epoch;
  long long limit;
  int members;
};

template <class R, int SH, bool GEN>
__global__ void __launch_bounds__(sweep_threads(GEN), GEN ? 4 : 1)
    k_sweep_persist(const DevFault<R>* __restrict__ fs, const Chunk* __restrict__ chunks, int nch,
                    double4* __restrict__ partial, int m_dt, const float4* __restrict__ wtab, int wtab_pieces,
                    float gen_ds_max, const int2* __restrict__ mm, int TM, const int2* __restrict__ fc,
                    bool ahead, const SweepBarrier bar, bool ring_evict_first) {
  __shared__ unsigned s_epoch, s_fail;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_epoch = *reinterpret_cast<volatile unsigned*>(bar.epoch);
    s_fail = 0u;
  }
  __syncthreads();
  const int c0 = static_cast<int>(static_cast<int64_t>(blockIdx.x) * nch / gridDim.x);
  const int c1 = static_cast<int>(static_cast<int64_t>(blockIdx.x + 1) * nch / gridDim.x);
  if (c1 > c0) {
    DevFault<R> none{};
    int k_stop = c1 - c0;
    const bool ok = sweep_chunks<R, SH, true, GEN>(none, fs, chunks, c0, c1 - c0, partial, m_dt, wtab, wtab_pieces,
                                                   gen_ds_max, kSpinLimit, false, &k_stop, ring_evict_first);
    if (!ok && tid == 0)
      for (int c = c0 + k_stop; c < c1; ++c) atomicOr(fs[chunks[c].pad].status, SBIEM_FLAG_WAIT);
  }
  // grid barrier (bounded)
  __syncthreads();
  if (tid == 0) {
    __threadfence();  // this CTA's partials before its arrival
    const unsigned ticket = atomicAdd(bar.count, 1u);
    if (ticket == gridDim.x - 1) {
      *reinterpret_cast<volatile unsigned*>(bar.count) = 0u;
      __threadfence();
      atomicAdd(bar.epoch, 1u);
    } else {
      bool released = false;
      for (long long q = 0; q < bar.limit; ++q) {
        if (*reinterpret_cast<volatile unsigned*>(bar.epoch) != s_epoch) {
          released = true;
          break;
        }
        __nanosleep(64);
      }
      if (!released) {
        s_fail = 1u;
        for (int r = 0; r < bar.members; ++r) atomicOr(fs[r].status, SBIEM_FLAG_WAIT);
      }
    }
    __threadfence();
  }
  __syncthreads();
  if (s_fail) return;
  for (int t = blockIdx.x * blockDim.x + tid; t < TM; t += gridDim.x * blockDim.x)
    finish_pair<R>(fs, mm, t, fc, nch, gridDim.x, partial, ahead);
}

// ------------------------------------------------------------ friction
// x = ln V solves g(x) = q(x) - eta e^x = 0 with q(x) = tau - sigma (c0 + a x),
// c0 = f0 + b ln(theta V0 / Dc) - a ln V0 (Eq. momentum plus radiation
// damping).  g is strictly decreasing and concave, so its root is unique and
// lies below the quasi-static root x_qs (q = 0).  Newton on g where friction
// dominates, on h(x) = x - ln(q/eta) (same root, increasing and convex)
// where radiation damping dominates (q > sigma a).  From either side a step
// of either form lands at or above the root, and from above it stays in
// [root, x): the iterates approach the root from above after the first step.
// Guards: a step above the bracket [lo, hi] (lo: largest point seen with
// g > 0, hi: smallest with g <= 0, initially x_qs) is replaced by
// bisection, and a step below lo by bisection too.
//
// FP64 is scarce on this part, so e^x is carried along the iteration: from
// V_prev when Newton starts at ln V_prev, then multiplied by e^dx from a
// Taylor series when |dx| <= 1/64 (truncation below 2e-19 relative), a full
// exp otherwise.  Returns iterations (negative: not converged); *xout = the
// root, *exout = e^root from the carried value (e^x (1 + dx) at the last,
// |dx| <= tol, step).  The caller takes a full exp every 1024th step, so the
// stored slip rate and its logarithm cannot drift apart.
__device__ __forceinline__ double exp_small(double d) {
  // e^d, |d| <= 1/64: Taylor polynomial of degree 7
  double p = 1.0 / 5040.0;
  p = fma(p, d, 1.0 / 720.0);
  p = fma(p, d, 1.0 / 120.0);
  p = fma(p, d, 1.0 / 24.0);
  p = fma(p, d, 1.0 / 6.0);
  p = fma(p, d, 0.5);
  p = fma(p, d, 1.0);
  return fma(p, d, 1.0);
}

// 1/d (d > 0) without an FP64 division, for the Newton steps and guards:
// the FP64 pipe is scarce on this part, and a division, like a conversion
// between FP64 and FP32, runs on it.  The seed is an FP32 reciprocal
// (rcp.approx) of d truncated to FP32 by integer operations on its bits
// (exponent rebiased by 1023 - 127 = 896, top 23 mantissa bits), widened
// back to FP64 the same way: relative error about 2^-22.  STEPS
// Newton-Raphson reciprocal steps r <- r + r (1 - d r) in FP64 follow, each
// squaring the relative error: about 6e-14 after one (a Newton step
// dx = g / g' taken with it converges as with the exact derivative), FP64
// rounding after two.  For d outside [1e-30, 1e30] (never met by the solve's
// quantities), d <= 0 and NaN, the division.
// Comparisons of doubles on the integer pipe: the FP64 pipe, which also
// executes FP64 comparisons and min/max, is what bounds the friction solve
// on this part.  The bit pattern of a double, with the magnitude bits
// flipped when the sign is set, orders like the value (-0 sorts just below
// +0, which the solve never tells apart; a NaN sorts beyond the infinity of
// its sign, so a NaN step still fails the convergence test and a NaN
// residual still ends in the iteration cap).
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool dgt(double a, double b) { return dkey(a) > dkey(b); }
__device__ __forceinline__ double dmin(double a, double b) { return dkey(a) < dkey(b) ? a : b; }
// |a| <= b and |a| < b for b >= 0 (false for a NaN a)
__device__ __forceinline__ bool dabs_le(double a, double b) {
  return (__double_as_longlong(a) & 0x7fffffffffffffffLL) <= __double_as_longlong(b);
}
__device__ __forceinline__ bool dabs_lt(double a, double b) {
  return (__double_as_longlong(a) & 0x7fffffffffffffffLL) < __double_as_longlong(b);
}
// FP32 -> FP64 on the integer pipe: exact for normal values, zeros,
// infinities and NaNs; FP32 subnormals (below 1.2e-38) become zero.
__device__ __forceinline__ double widen(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sgn = static_cast<unsigned long long>(u & 0x80000000u) << 32;
  if (e == 0u) return __longlong_as_double(static_cast<long long>(sgn));
  const unsigned long long ex = e == 0xffu ? 0x7ffull : static_cast<unsigned long long>(e + 896u);
  return __longlong_as_double(
      static_cast<long long>(sgn | (ex << 52) | (static_cast<unsigned long long>(u & 0x7fffffu) << 29)));
}

template <int STEPS>
__device__ __forceinline__ double rcp_nr(double d) {
  const long long db = __double_as_longlong(d);
  if (!(db >= __double_as_longlong(1e-30) && db <= __double_as_longlong(1e30))) return 1.0 / d;
  const unsigned hi = static_cast<unsigned>(__double2hiint(d)), lo = static_cast<unsigned>(__double2loint(d));
  const unsigned fb = __funnelshift_l(lo, hi - 0x38000000u, 3);  // FP32 bits of d, truncated
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(fb)));
  const unsigned rb = __float_as_uint(rf);
  double r = __hiloint2double(static_cast<int>((rb >> 3) + 0x38000000u), static_cast<int>(rb << 29));
#pragma unroll
  for (int k = 0; k < STEPS; ++k) r = fma(r, fma(-d, r, 1.0), r);
  return r;
}

__device__ __forceinline__ int solve_lnV(double tau, double sig, double c0, double a, double eta, double reta,
                                          double x0, double ex0, double xguess, double tol, int maxit,
                                          double* xout, double* exout) {
  const double sa = sig * a;
  // x_qs: only the guards below need it, so its division overlaps the
  // first residual (a start above x_qs has g < 0 and steps down)
  double hi = dmin((tau - sig * c0) * rcp_nr<2>(sa), 700.0);
  double lo = -CUDART_INF;
  // a learned guess is used when it is finite, below x_qs and calls for a
  // substantial change (|guess - ln V_prev| >= 0.1, where the previous slip
  // rate is a poor start); otherwise the previous slip rate starts Newton
  const bool use_guess = isfinite(xguess) && !dgt(xguess, hi) && !dabs_lt(xguess - x0, 0.1);
  double x = x0, ex = ex0;
  if (use_guess) {
    x = xguess;
    ex = exp(x);
  }
  for (int it = 1; it <= maxit; ++it) {
    const double e = eta * ex;
    const double q = tau - sig * fma(a, x, c0);
    const double g = q - e;
    if (dgt(g, 0.0)) lo = x; else hi = dmin(hi, x);
    double dx;
    if (dgt(q, sa)) dx = -q * (x - log(q * reta)) * rcp_nr<1>(q + sa);
    else dx = g * rcp_nr<1>(e + sa);
    if (dabs_le(dx, tol)) {
      *xout = x + dx;
      *exout = ex * (1.0 + dx);
      return it;
    }
    double xn = x + dx;
    // keep Newton points within tol of the bracket: roots next to the
    // quasi-static bound (vanishing radiation damping) land on it up to rounding
    if (dgt(xn, hi + tol) || dgt(lo - tol, xn)) {
      xn = (__double_as_longlong(lo) != __double_as_longlong(-CUDART_INF)) ? 0.5 * (lo + hi) : hi;
      dx = xn - x;
    }
    ex = dabs_le(dx, 0.015625) ? ex * exp_small(dx) : exp(xn);
    x = xn;
  }
  *xout = x;
  *exout = ex;
  return -maxit;
}

// MLP: the variant that can evaluate the learned initial guess (compiled
// separately so the plain solve stays small in the instruction cache).
template <class R, bool MLP>
__device__ __forceinline__ void newton_body(const DevFault<R>& f, int pass, double dt) {
  // each warp (block) takes newton_epw elements: fewer than 32 spreads the
  // FP64 work of small faults over more SM partitions
  const int epw = f.newton_epw;
  const int i = threadIdx.x < epw ? blockIdx.x * epw + threadIdx.x : f.N;
  // launched early behind the spectral pass: everything it reads is written
  // by the kernels before it
  pdl_trigger();
  pdl_wait();
  // one read of the status word per block: other blocks may set it while
  // this one runs, and the decision must be uniform across the warp
  __shared__ unsigned s_skip;
  if (threadIdx.x == 0) s_skip = *f.status;
  const bool have = i < f.N;
  // every per-element input is loaded here, unconditionally and beside the
  // status read: one memory latency before the arithmetic (lanes without an
  // element read element 0; a value a branch below does not use costs only
  // its bytes)
  const int ic = have ? i : 0;
  const double ld_V = f.V[ic], ld_V1 = f.V1[ic], ld_Dc = f.Dc[ic], ld_rDc = f.rDc[ic], ld_th = f.th[ic];
  const double ld_psi = f.psi[ic], ld_thd = f.thd[ic], ld_thd1 = f.thd1[ic];
  const Cx<R> y = f.y[ic];
  const double ld_tau0 = f.tau0[ic], ld_taur = f.taur[ic], ld_sig0 = f.sig0[ic];
  const double ld_xV = f.xV[ic], ld_x1 = f.x1[ic];
  const bool ld_presc = f.presc[ic] != 0;
  const double ld_a = f.a[ic], ld_b = f.b[ic], ld_lvd = f.lvd[ic], ld_Vp = f.Vp[ic];
  const double ld_kappa = f.kappa[ic], ld_delta = f.delta[ic];
  const double t_now = *f.t;
  const long long steps = *f.steps_done;
  __syncthreads();
  if (s_skip) return;
  unsigned flags = 0u;
  int iters = 0;
  // per-element quantities of the solve (dummies on lanes without an element,
  // which still take part in the warp-wide network evaluation)
  double vb = 0.0, Dc = 1.0, rDc = 1.0, thp = 1.0, psip = 0.0, tau = 0.0, sig = 1.0, xstart = 0.0, a = 0.01,
         c0 = 0.0;
  // every 1024th step recomputes ln theta and e^x in full (see below)
  const bool resync_off = (steps & 1023) != 0;
  bool solve = false;
  if (have) {
    // pass slip rate: the committed one, then the mean of committed and pass-1
    vb = (pass == 1) ? ld_V : 0.5 * (ld_V + ld_V1);
    Dc = ld_Dc;
    rDc = ld_rDc;
    const double th0 = ld_th;
    const double rth0 = rcp_nr<1>(th0);  // off the chain: used only in the series branch
    bool series = false;
    if (f.state_law == 0) {
      // aging law integrated at constant Vbar: theta e^{-u} + dt phi(u),
      // phi(u) = (1 - e^{-u})/u, u = Vbar dt / Dc
      const double u = vb * dt * rDc;
      if (dgt(1e-4, u)) {
        // series of phi to u^3 (truncation below u^4/120 < 1e-18); with
        // e^{-u} = 1 - u phi the update is theta (1 + z), z = phi (dt/theta - u)
        const double phi = fma(fma(fma(-u, 1.0 / 24.0, 1.0 / 6.0), u, -0.5), u, 1.0);
        const double z = phi * fma(dt, rth0, -u);
        thp = fma(th0, z, th0);
        // every 1024th step takes the full log, so ln theta and theta, kept
        // side by side, cannot drift apart by accumulated rounding
        if (dabs_lt(z, 1e-3) && resync_off) {
          // ln theta' = ln theta + log1p(z), series to z^6 (truncation below
          // |z|^7/7 < 2e-22)
          double l = -1.0 / 6.0;
          l = fma(l, z, 1.0 / 5.0);
          l = fma(l, z, -0.25);
          l = fma(l, z, 1.0 / 3.0);
          l = fma(l, z, -0.5);
          l = fma(l, z, 1.0);
          psip = fma(l, z, ld_psi);
          series = true;
        }
      } else {
        const double em = expm1(-u);
        const double eu = u < 1.0 ? 1.0 + em : exp(-u);
        thp = fma(th0, eu, dt * (-em / u));
      }
    } else {
      const double thdb = (pass == 1) ? ld_thd : 0.5 * (ld_thd + ld_thd1);
      thp = th0 + thdb * dt;
      if (!(thp > 0.0)) flags |= SBIEM_FLAG_STATE;
    }
    if (!series) psip = log(thp);
    const double t_end = t_now + dt;
    if constexpr (sizeof(R) == 4) {
      tau = ld_tau0 + ld_taur * t_end + widen(y.x);
      sig = ld_sig0 + widen(y.y);
    } else {
      tau = ld_tau0 + ld_taur * t_end + static_cast<double>(y.x);
      sig = ld_sig0 + static_cast<double>(y.y);
    }
    xstart = (pass == 1) ? ld_xV : ld_x1;
    if (!ld_presc) {
      if (!(sig > 0.0)) flags |= SBIEM_FLAG_OPENING;
      solve = flags == 0u;
      a = ld_a;
      // f0 + a (x - ln V0) + b ln(theta V0 / Dc) = c0 + a x
      c0 = f.f0 + ld_b * (psip + ld_lvd) - a * f.lnV0;
    }
  }
  double xguess = CUDART_NAN;
  if (MLP && f.mlp) {
    // The guess is used only when it lies at least 0.1 from ln V_prev, and
    // the first Newton step from ln V_prev bounds the distance to the root
    // (from either side a step lands at or above the root, and from above
    // the root lies within it).  A warp whose every first step is shorter
    // than 0.1 would land on the same roots without the guess: it skips the
    // network (warp-uniform, as the network's tiles span the warp).
    bool need = false;
    if (have && solve) {
      const double ex0 = (pass == 1) ? ld_V : ld_V1;
      const double e = f.eta * ex0, q = tau - sig * fma(a, xstart, c0), sa = sig * a;
      // (a threshold test: the FP32 reciprocal is enough)
      const double dx0 =
          dgt(q, sa) ? -q * (xstart - log(q * f.reta)) * rcp_nr<0>(q + sa) : (q - e) * rcp_nr<0>(e + sa);
      need = !dabs_lt(dx0, 0.1);
    }
    if (__any_sync(0xffffffffu, need)) {
      const float feat[kMlpIn] = {static_cast<float>(xstart), static_cast<float>(psip),
                                  static_cast<float>(tau / sig), static_cast<float>(a),
                                  static_cast<float>(have ? ld_b : 0.015)};
      xguess = xstart + static_cast<double>(mlp_residual_warp(*f.mlp, feat));
    }
  }
  if (have) {
    double x, exn = -1.0;  // exn: e^x carried by the solve (< 0: not solved)
    if (ld_presc) {
      x = xstart;  // ln V_presc, kept in ln V since creation
    } else if (!solve) {
      x = ld_xV;
    } else {
      // e^xstart: the slip rate whose log starts Newton
      const double ex0 = (pass == 1) ? ld_V : ld_V1;
      const int it =
          solve_lnV(tau, sig, c0, a, f.eta, f.reta, xstart, ex0, xguess, f.newton_tol, f.newton_maxit, &x, &exn);
      if (it < 0) flags |= SBIEM_FLAG_NEWTON;
      iters = it < 0 ? -it : it;
      if (it > 0 && f.harvest) {
        const unsigned long long k = atomicAdd(f.harvest_count, 1ull);
        if (k < static_cast<unsigned long long>(f.harvest_cap)) {
          float* row = f.harvest + 6 * k;
          row[0] = static_cast<float>(xstart);
          row[1] = static_cast<float>(psip);
          row[2] = static_cast<float>(tau / sig);
          row[3] = static_cast<float>(a);
          row[4] = static_cast<float>(ld_b);
          row[5] = static_cast<float>(x);
        }
      }
    }
    const double Vn = ld_presc ? ld_Vp : ((exn > 0.0 && resync_off) ? exn : exp(x));
    const double thd_new = 1.0 - thp * Vn * rDc;
    if (pass == 1) {
      f.V1[i] = Vn;
      f.x1[i] = x;
      f.thd1[i] = thd_new;
      if (f.zin2) {
        // FP32 input of the pass-2 FFT
        const double v2 = 0.5 * (ld_V + Vn);
        f.zin2[i] = make_float2(static_cast<float>(v2), static_cast<float>(ld_kappa * v2));
      }
    } else {
      f.V2[i] = Vn;
      f.x2[i] = x;
      f.psi2[i] = psip;
      f.th2[i] = thp;
      f.thd2[i] = thd_new;
      f.delta2[i] = ld_delta + vb * dt;
    }
  }
  // warp-level aggregation of flags and iteration counts, one atomic per warp
  unsigned fl = flags;
  int im = iters;
  unsigned long long is = static_cast<unsigned long long>(iters);
  unsigned ns = (have && solve && !ld_presc) ? 1u : 0u;  // Newton solves (a guess or plain start)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fl |= __shfl_xor_sync(0xffffffffu, fl, o);
    im = max(im, __shfl_xor_sync(0xffffffffu, im, o));
    is += __shfl_xor_sync(0xffffffffu, is, o);
    ns += __shfl_xor_sync(0xffffffffu, ns, o);
  }
  if (threadIdx.x == 0) {
    if (fl) atomicOr(f.status, fl);
    if (im) atomicMax(f.it_max, im);
    if (is) atomicAdd(f.it_sum, is);
    if (f.it_total && ns) {
      // running totals over every solve since the last reset (sbiem_newton_totals)
      atomicAdd(f.it_total, is);
      atomicAdd(f.it_total + 1, static_cast<unsigned long long>(ns));
    }
  }
}

template <class R, bool MLP>
__global__ void __launch_bounds__(32) k_newton(const __grid_constant__ DevFault<R> f, int pass, double dt) {
  newton_body<R, MLP>(f, pass, dt);
}

template <class R>
__global__ void __launch_bounds__(32) k_newton_b(const DevFault<R>* __restrict__ fs, int pass, int m_dt) {
  const DevFault<R>& f = fs[blockIdx.y];
  newton_body<R, true>(f, pass, m_dt * f.dt_min);
}

// ------------------------------------------------------------- commit
template <class R>
__device__ __forceinline__ void commit_body(const DevFault<R>& f, int m_dt, double dt, int lag_p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // launched early behind the pass-2 Newton: static tables first, then the wait
  const bool md0 = i < f.nmodes;
  const int Rn0 = md0 ? f.Rn[i] : 0;
  const int64_t roff0 = md0 ? f.ring_off[i] : 0;
  pdl_wait();
  // every load first (one memory latency), the status decision, then stores
  const unsigned status = *f.status;
  const bool el = i < f.N, md = i < f.nmodes;
  double v = 0.0, x2 = 0.0, psi2 = 0.0, th2 = 0.0, thd2 = 0.0, d2 = 0.0, kap = 0.0;
  if (el) {
    v = f.V2[i];
    x2 = f.x2[i];
    psi2 = f.psi2[i];
    th2 = f.th2[i];
    thd2 = f.thd2[i];
    d2 = f.delta2[i];
    if (f.zin1) kap = f.kappa[i];
  }
  double2 U = make_double2(0.0, 0.0), Q = U, D = U, K = U, T = U, Nn = U, w1 = U, w0 = U;
  int Rn = 0, h = 0;
  int64_t roff = 0;
  if (md) {
    U = f.U2f ? make_double2(f.U2f[i].x, f.U2f[i].y) : f.U2[i];
    Q = f.Q2f ? make_double2(f.Q2f[i].x, f.Q2f[i].y) : f.Q2[i];
    D = f.dhat[i];
    K = f.khat[i];
    Rn = Rn0;
    roff = roff0;
    h = f.head[i];
    if (lag_p >= 0) {
      T = f.BT[i];
      Nn = f.BN[i];
      w1 = f.w0pow[static_cast<size_t>(i) * kPow2Slots + lag_p + 1];
      w0 = f.w0pow[static_cast<size_t>(i) * kPow2Slots + lag_p];
    }
  }
  if (status) return;
  if (el) {
    f.V[i] = v;
    f.xV[i] = x2;
    f.psi[i] = psi2;
    f.th[i] = th2;
    f.thd[i] = thd2;
    f.delta[i] = d2;
    if (f.zin1) f.zin1[i] = make_float2(static_cast<float>(v), static_cast<float>(kap * v));
  }
  if (md) {
    D.x += dt * U.x;
    D.y += dt * U.y;
    K.x += dt * Q.x;
    K.y += dt * Q.y;
    f.dhat[i] = D;
    f.khat[i] = K;
    if (f.dhat32) {
      f.dhat32[i] = make_float2(static_cast<float>(D.x), static_cast<float>(D.y));
      f.khat32[i] = make_float2(static_cast<float>(K.x), static_cast<float>(K.y));
    }
    // the value the ring holds (FP32 in the precision form)
    double2 sT = U, sN = Q;
    if (Rn > 0) {
      Slot<R> sl;
      if constexpr (sizeof(R) == 8) {
        sl.t = U;
        sl.n = Q;
      } else {
        sl = make_float4(static_cast<float>(U.x), static_cast<float>(U.y), static_cast<float>(Q.x),
                         static_cast<float>(Q.y));
        sT = make_double2(sl.x, sl.y);
        sN = make_double2(sl.z, sl.w);
      }
      if (m_dt == 1) {
        h = (h == 0) ? Rn - 1 : h - 1;
        f.ring[roff + h] = sl;
      } else {
        // the m_dt copies were written by k_push_multi; move the head
        h = static_cast<int>(((h - static_cast<int64_t>(m_dt)) % Rn + Rn) % Rn);
      }
      f.head[i] = h;
    }
    if (lag_p >= 0) {
      // overlapped form: the next step (same m_dt) sees this step's slot at
      // lags m_dt .. 2 m_dt - 1 and the older slots through BT/BN
      if (Rn > 0) {
        const double wT = w1.x - w0.x, wN = w1.y - w0.y;
        T.x = fma(wT, sT.x, T.x);
        T.y = fma(wT, sT.y, T.y);
        Nn.x = fma(wN, sN.x, Nn.x);
        Nn.y = fma(wN, sN.y, Nn.y);
      }
      f.AT[i] = T;
      f.AN[i] = Nn;
      if (f.AT32) {
        f.AT32[i] = make_float2(static_cast<float>(T.x), static_cast<float>(T.y));
        f.AN32[i] = make_float2(static_cast<float>(Nn.x), static_cast<float>(Nn.y));
      }
    }
  }
  if (i == 0) {
    *f.steps_done += 1;
    *f.t += dt;
  }
}

template <class R>
__global__ void k_commit(const __grid_constant__ DevFault<R> f, int m_dt, double dt, int lag_p) {
  commit_body<R>(f, m_dt, dt, lag_p);
}

template <class R>
__global__ void k_commit_b(const DevFault<R>* __restrict__ fs, int m_dt, int lag_p) {
  const DevFault<R>& f = fs[blockIdx.y];
  commit_body<R>(f, m_dt, m_dt * f.dt_min, lag_p);
}

// Push of m_dt > 1 copies of this step's spectra (a step of m_dt dt_min,
// Sec. 3.3 last paragraph on the dt_min grid): the logical slots
// i < min(m_dt, R_n) after the push hold the value.  Runs before k_commit,
// which moves the heads.
template <class R>
__global__ void k_push_multi(DevFault<R> f, int m_dt) {
  if (*f.status) return;
  for (int c = blockIdx.x; c < f.nchunks; c += gridDim.x) {
    const Chunk cd = f.chunks[c];
    const int n = cd.mode;
    const int Rn = f.Rn[n];
    const int cnt = min(m_dt, Rn);
    if (cd.i0 >= cnt) continue;
    const int hn = static_cast<int>(((f.head[n] - static_cast<int64_t>(cnt)) % Rn + Rn) % Rn);
    const double2 U = f.U2f ? make_double2(f.U2f[n].x, f.U2f[n].y) : f.U2[n];
    const double2 Q = f.Q2f ? make_double2(f.Q2f[n].x, f.Q2f[n].y) : f.Q2[n];
    Slot<R> v;
    if constexpr (sizeof(R) == 8) {
      v.t = U;
      v.n = Q;
    } else {
      v = make_float4(static_cast<float>(U.x), static_cast<float>(U.y), static_cast<float>(Q.x),
                      static_cast<float>(Q.y));
    }
    Slot<R>* ring = f.ring + f.ring_off[n];
    const int64_t iend = min(cd.i1, static_cast<int64_t>(cnt));
    for (int64_t i = cd.i0 + threadIdx.x; i < iend; i += blockDim.x) {
      int64_t pos = hn + i;
      if (pos >= Rn) pos -= Rn;
      ring[pos] = v;
    }
  }
}

// w0pow[n][p] = sum_{j < min(2^p, M_n)} w_{n,j} (FP64, both fields): the
// weight of a current interval of 2^p dt_min.  One block per mode; segment
// [2^(p-1), 2^p) summed by a fixed-order block reduction, so the result does
// not depend on scheduling.
template <class R>
__global__ void k_weight_pow2(const W2<R>* w, const int64_t* w_off, const int32_t* Mn, int nmodes, double2* out,
                              float2* c0, double S, double mu, double dt_min) {
  __shared__ double shT[32], shN[32];
  const int n = blockIdx.x;
  if (n >= nmodes) return;
  const int M = Mn[n];
  const W2<R>* wn = w + w_off[n];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double run_T = 0.0, run_N = 0.0;
  for (int p = 0; p < kPow2Slots; ++p) {
    const int64_t lo = p == 0 ? 0 : (static_cast<int64_t>(1) << (p - 1));
    const int64_t hi = min(static_cast<int64_t>(1) << p, static_cast<int64_t>(M));
    double sT = 0.0, sN = 0.0;
    for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
      sT += static_cast<double>(wn[j].x);
      sN += static_cast<double>(wn[j].y);
    }
    sT = warp_sum(sT);
    sN = warp_sum(sN);
    if (lane == 0) {
      shT[wid] = sT;
      shN[wid] = sN;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 0; q < nw; ++q) {
        run_T += shT[q];
        run_N += shN[q];
      }
      out[static_cast<size_t>(n) * kPow2Slots + p] = make_double2(run_T, run_N);
      if (c0) {
        const double sdt = S * dt_min * static_cast<double>(static_cast<int64_t>(1) << p);
        c0[static_cast<size_t>(n) * kPow2Slots + p] =
            make_float2(static_cast<float>(sdt + mu * run_T), static_cast<float>(sdt + mu * run_N));
      }
    }
    __syncthreads();
  }
}

// Copy the ring slots a push of m_dt copies overwrites (positions
// head - min(m_dt, R) .. head - 1) to or from the undo buffer (same layout as
// the ring).  dir = 0: save, 1: restore.
template <class R>
__global__ void k_ring_undo(DevFault<R> f, int m_dt, Slot<R>* undo, int dir) {
  for (int c = blockIdx.x; c < f.nchunks; c += gridDim.x) {
    const Chunk cd = f.chunks[c];
    const int n = cd.mode;
    const int Rn = f.Rn[n];
    const int cnt = min(m_dt, Rn);
    if (cd.i0 >= cnt) continue;
    const int hn = static_cast<int>(((f.head[n] - static_cast<int64_t>(cnt)) % Rn + Rn) % Rn);
    Slot<R>* ring = f.ring + f.ring_off[n];
    Slot<R>* u = undo + f.ring_off[n];
    const int64_t iend = min(cd.i1, static_cast<int64_t>(cnt));
    for (int64_t i = cd.i0 + threadIdx.x; i < iend; i += blockDim.x) {
      int64_t pos = hn + i;
      if (pos >= Rn) pos -= Rn;
      if (dir == 0) u[i] = ring[pos];
      else ring[pos] = u[i];
    }
  }
}

// The ring slot a step of one dt_min overwrites in each mode (the slot
// before the head): saved into buf[n] (dir 0) or put back (dir 1), so that
// a step taken only to time it can be undone with the state snapshot.
template <class R>
__global__ void k_slot_swap(DevFault<R> f, Slot<R>* buf, int dir) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= f.nmodes) return;
  const int Rn = f.Rn[n];
  if (Rn <= 0) return;
  const int h = f.head[n];
  Slot<R>* slot = f.ring + f.ring_off[n] + (h == 0 ? Rn - 1 : h - 1);
  if (dir == 0) buf[n] = *slot;
  else *slot = buf[n];
}

template <class R>
void launch_slot_swap(const DevFault<R>& f, void* buf, int dir, cudaStream_t st) {
  k_slot_swap<R><<<(f.nmodes + 255) / 256, 256, 0, st>>>(f, static_cast<Slot<R>*>(buf), dir);
}
template void launch_slot_swap<double>(const DevFault<double>&, void*, int, cudaStream_t);
template void launch_slot_swap<float>(const DevFault<float>&, void*, int, cudaStream_t);

// max_i |a_i - b_i| into *out (one block).
__global__ void k_maxdiff(const double* a, const double* b, int n, double* out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(a[i] - b[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *out = m;
  }
}

// ------------------------------------------------------------- weights
// (C^T(s), C^N(s)) from the piecewise Chebyshev table (Clenshaw recurrence).
__device__ __forceinline__ double2 cheb_kernels(const double* __restrict__ cheb, int npieces, int deg, double h,
                                                double s) {
  int p = static_cast<int>(s / h);
  p = min(p, npieces - 1);
  const double t = 2.0 * (s - p * h) / h - 1.0;
  const double* c = cheb + static_cast<size_t>(p) * (deg + 1) * 2;
  double bT1 = 0.0, bT2 = 0.0, bN1 = 0.0, bN2 = 0.0;
  for (int kk = deg; kk >= 1; --kk) {
    const double tT = 2.0 * t * bT1 - bT2 + c[2 * kk];
    const double tN = 2.0 * t * bN1 - bN2 + c[2 * kk + 1];
    bT2 = bT1;
    bT1 = tT;
    bN2 = bN1;
    bN1 = tN;
  }
  return make_double2(t * bT1 - bT2 + c[0], t * bN1 - bN2 + c[1]);
}

// Six-point Gauss-Legendre rule on [-1, 1] (nodes +-x, weights w): the
// interval weights of the exact quadrature option.  An interval spans at
// most pi/4 in s and the kernels oscillate at most at 1/r in s, so the
// rule's error term (6!)^4 / (13 (12!)^3) (h w / 2)^12 stays below 1e-17.
__constant__ double kGL6x[3] = {0.2386191860831969086305017, 0.6612093864662645136613996,
                                0.9324695142031520278123016};
__constant__ double kGL6w[3] = {0.4679139345726910473898703, 0.3607615730481386075698335,
                                0.1713244923791703450402961};

// Weights of lag j of mode n: quadrature 0 (midpoint rule, Sec. 3.3):
// w_{n,j} = dt_min C(k_n, (j + 1/2) dt_min); quadrature 1: the integral of
// C(k_n, tau) over [j dt_min, (j + 1) dt_min] (six-point Gauss-Legendre on
// the interval).  MT, MN (may be NULL): the shear and normal kernels' own
// windows when they are cut at two planes (Sec. 3.1); a field's weights are
// zero past its own.
template <class R>
__global__ void k_weights(W2<R>* w, const int64_t* w_off, const int32_t* Mn, int nmodes, double L,
                          double cs, double dt, const double* __restrict__ cheb, int npieces, int deg,
                          double h, const int32_t* MT, const int32_t* MN, int quadrature) {
  const int n = blockIdx.x;
  if (n == 0 || n >= nmodes) return;
  const double k = kTwoPi * n / L;
  const double ds = cs * k * dt;
  const int M = Mn[n];
  const int MTn = MT ? MT[n] : M, MNn = MN ? MN[n] : M;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    double2 c;
    if (quadrature == 0) {
      c = cheb_kernels(cheb, npieces, deg, h, ds * (j + 0.5));
    } else {
      c = make_double2(0.0, 0.0);
      for (int q = 0; q < 3; ++q) {
        const double2 a = cheb_kernels(cheb, npieces, deg, h, ds * (j + 0.5 * (1.0 - kGL6x[q])));
        const double2 b = cheb_kernels(cheb, npieces, deg, h, ds * (j + 0.5 * (1.0 + kGL6x[q])));
        c.x += 0.5 * kGL6w[q] * (a.x + b.x);
        c.y += 0.5 * kGL6w[q] * (a.y + b.y);
      }
    }
    W2<R> out;
    out.x = j < MTn ? static_cast<R>(dt * c.x) : R(0);
    out.y = j < MNn ? static_cast<R>(dt * c.y) : R(0);
    w[w_off[n] + j] = out;
  }
}

// ------------------------------------------------------------- utilities
__global__ void k_pack(int N, const double* x, const double* y, const double* ymul, double2* z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double yi = 0.0;
  if (y) yi = y[i] * (ymul ? ymul[i] : 1.0);
  z[i] = make_double2(x[i], yi);
}

__global__ void k_unpack(int N, const double2* Z, double2* X, double2* Y) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n > N / 2) return;
  const double2 a = Z[n], c = Z[(N - n) & (N - 1)];
  if (X) X[n] = make_double2(0.5 * (a.x + c.x), 0.5 * (a.y - c.y));
  if (Y) Y[n] = make_double2(0.5 * (a.y + c.y), -0.5 * (a.x - c.x));
}

__global__ void k_d2(int N, double L, double2* Z) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int m = n <= N / 2 ? n : N - n;
  const double k = kTwoPi * m / L;
  Z[n].x *= -k * k;
  Z[n].y *= -k * k;
}

__global__ void k_real_part(int N, const double2* z, double* x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) x[i] = z[i].x;
}

// ------------------------------------------------------------- launchers
FftGeom make_geom(int N, int elem_bytes) {
  FftGeom g{};
  g.N = N;
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  g.lgN1 = (lg + 1) / 2;
  g.lgN2 = lg - g.lgN1;
  g.N1 = 1 << g.lgN1;
  g.N2 = 1 << g.lgN2;
  // B rows or columns per CTA: 32 contiguous bytes per global segment; for
  // large N fewer, down to one, while a pass would have fewer than 256 CTAs
  // (the arrays are then L2 resident, and CTAs on every SM shorten the
  // latency-bound pass)
  const int B = elem_bytes >= 32 ? 1 : 32 / elem_bytes;
  g.Bc = B < g.N1 ? B : g.N1;
  g.Br = B < g.N2 ? B : g.N2;
  if (N >= 32768) {
    while (g.Bc > 1 && g.N1 / g.Bc < 256) g.Bc /= 2;
    while (g.Br > 1 && g.N2 / g.Br < 256) g.Br /= 2;
  }
  auto threads = [](int work) {
    int t = work;
    if (t > 256) t = 256;
    if (t < 32) t = 32;
    return t;
  };
  g.tc = threads(g.Bc * g.N2 / 2);
  g.tr = threads(g.Br * g.N1 / 2);
  return g;
}

template <class R>
static size_t col_smem(const FftGeom& g) { return (static_cast<size_t>(g.Bc) * g.N2 + g.N2 / 2) * sizeof(Cx<R>); }
template <class R>
static size_t row_smem(const FftGeom& g) { return (static_cast<size_t>(g.Br) * g.N1 + g.N1 / 2) * sizeof(Cx<R>); }

// Opt in to dynamic shared memory.  The attribute belongs to the function,
// not to a handle, and handles of different N launch the same kernels, so it
// is raised to the device's opt-in limit (never lowered to one handle's
// need); the launch's own size still decides occupancy.
template <class K>
static void allow_smem(K kernel, size_t bytes) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, kernel);
  const int avail = optin - static_cast<int>(fa.sharedSizeBytes);
  if (static_cast<int>(bytes) <= avail)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, avail);
}


static size_t fused_smem(int N) { return static_cast<size_t>(N + N / 2) * sizeof(float2); }
// cluster pass: column and row buffers (N/C each) and the N2/2 + N1/2 sub-table twiddles
static size_t cluster_smem(int N, int C) {
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  const int N1 = 1 << (lg / 2), N2 = 1 << (lg - lg / 2);
  const size_t per = static_cast<size_t>(N / C);
  return (4 * per + N1 / 2 + N2 / 2) * sizeof(float2) + per * sizeof(ModeIn);
}

// fn(std::integral_constant<int, log2 N>) for the sizes of the one-launch
// FP32 spectral pass (16 <= N <= kFusedMaxN).
template <class F>
static void with_lgn(int N, F&& fn) {
  switch (31 - __builtin_clz(static_cast<unsigned>(N))) {
    case 4: fn(std::integral_constant<int, 4>{}); break;
    case 5: fn(std::integral_constant<int, 5>{}); break;
    case 6: fn(std::integral_constant<int, 6>{}); break;
    case 7: fn(std::integral_constant<int, 7>{}); break;
    case 8: fn(std::integral_constant<int, 8>{}); break;
    case 9: fn(std::integral_constant<int, 9>{}); break;
    case 10: fn(std::integral_constant<int, 10>{}); break;
    case 11: fn(std::integral_constant<int, 11>{}); break;
    case 12: fn(std::integral_constant<int, 12>{}); break;
    case 13: fn(std::integral_constant<int, 13>{}); break;
    case 14: fn(std::integral_constant<int, 14>{}); break;
    default: break;
  }
}
static_assert(kFusedMaxN == 1 << 14 && kClusterMinN == 1 << 11, "with_lgn covers the one-launch pass sizes");

// Launch with the attributes of the pass kernels: a cluster of `cluster`
// CTAs (> 1), programmatic dependent launch behind the stream's previous
// kernel (early; the kernel waits in pdl_wait()), and an event that fires
// once every CTA has started (started, may be null: the overlapped step
// dispatches its side-branch sweep only then, so that the sweep never takes
// the SMs ahead of the pass's first kernel).
template <class... Args>
static void launch_attr(void (*kernel)(Args...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int cluster,
                        bool early, cudaEvent_t started, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[3];
  int na = 0;
  if (cluster > 1) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = cluster;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  if (early) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (started) {
    at[na].id = cudaLaunchAttributeProgrammaticEvent;
    at[na].val.programmaticEvent.event = started;
    at[na].val.programmaticEvent.flags = 0;
    at[na].val.programmaticEvent.triggerAtBlockStart = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Cluster launch of the FP32 spectral pass (one cluster per fault).
template <class... Args>
static void launch_cluster_kernel(void (*kernel)(Args...), int clusters, int N, int C, cudaStream_t st,
                                  bool early, cudaEvent_t started, Args... args) {
  launch_attr(kernel, dim3(C * clusters), dim3(N / (kClusterEPT * C)), cluster_smem(N, C), st, C, early, started,
              args...);
}

// Launch that may start before its predecessor on the stream finishes
// (programmatic dependent launch; the kernel waits in pdl_wait()).
template <class... Args>
static void launch_early(void (*kernel)(Args...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                         Args... args) {
  launch_attr(kernel, grid, block, smem, st, 1, true, static_cast<cudaEvent_t>(nullptr), args...);
}

// The spectral part of a pass (forward FFT, assembly, inverse FFT of Sec. 3.3 step (2); the predictor in the
// FP64 four-kernel form): one launch, or the four-step kernels.
template <class R>
void launch_spectral(const DevFault<R>& f, int pass, int m_dt, cudaStream_t st, cudaEvent_t started) {
  const FftGeom& g = f.g;
  const double dt = m_dt * f.dt_min;
  if constexpr (sizeof(R) == 4) {
    if (f.N <= kFusedMaxN) {
      with_lgn(f.N, [&](auto lg) {
        constexpr int LG = decltype(lg)::value;
        // pass 2 starts early behind the pass-1 Newton
        if constexpr ((1 << LG) >= kClusterMinN) {
          launch_cluster_kernel(k_spectral_cluster<LG, kClusterEPT>, 1, f.N, cluster_ctas(f.N), st, pass == 2,
                                started, f, pass, m_dt, dt);
        } else {
          launch_attr(k_spectral_fused<LG>, dim3(1), dim3(f.N / 8), fused_smem(f.N), st, 1, pass == 2, started, f,
                      pass, m_dt, dt);
        }
      });
      return;
    }
  }
  const size_t cs = col_smem<R>(g), rs = row_smem<R>(g);
  auto kfa = k_col<R, false, PRO_PASS>;
  auto kfb = k_row<R, false>;
  auto kia = k_col<R, true, PRO_ASSEMBLE>;
  auto kib = k_row<R, true>;
  launch_attr(kfa, dim3(g.N1 / g.Bc), dim3(g.tc), cs, st, 1, false, started, g, static_cast<const Cx<R>*>(f.tw),
              static_cast<const Cx<R>*>(nullptr), f.zt, f, pass, m_dt, dt);
  kfb<<<g.N2 / g.Br, g.tr, rs, st>>>(g, f.tw, f.zt, f.Z, R(1), f.status);
  kia<<<g.N1 / g.Bc, g.tc, cs, st>>>(g, f.tw, nullptr, f.zt, f, pass, m_dt, dt);
  kib<<<g.N2 / g.Br, g.tr, rs, st>>>(g, f.tw, f.zt, f.y, R(1.0 / g.N), f.status);
}

// The Newton part of a pass (state predictor and friction solve, Sec. 3.3), started early behind the spectral part.
template <class R>
void launch_newton(const DevFault<R>& f, int pass, int m_dt, cudaStream_t st) {
  const double dt = m_dt * f.dt_min;
  launch_early(f.mlp ? k_newton<R, true> : k_newton<R, false>, dim3((f.N + f.newton_epw - 1) / f.newton_epw),
               dim3(32), 0, st, f, pass, dt);
}

template <class R>
void launch_pass(const DevFault<R>& f, int pass, int m_dt, cudaStream_t st) {
  launch_spectral<R>(f, pass, m_dt, st);
  launch_newton<R>(f, pass, m_dt, st);
}

template <class R>
void launch_history_atomic(const DevFault<R>& f, int m_dt, int grid, cudaStream_t st) {
  if (f.nchunks == 0) return;
  const int warps = kHistThreads / 32;
  const int need = (f.nchunks + warps - 1) / warps;
  const int gr = grid < need ? grid : need;
  k_history_t<R, false><<<gr, kHistThreads, 0, st>>>(f, nullptr, f.chunks, f.nchunks, f.work, m_dt);
}

// Dynamic shared memory of the sweep: its stages.
template <class R, int SH>
static size_t sweep_smem() {
  return SweepCfg<R, SH>::kStages * sweep_stage_bytes<R, SH>();
}

// k_sweep<R, SH, BATCH, GEN> with GEN only where R is float.
template <class R, int SH, bool BATCH, bool GEN>
static auto sweep_kernel() {
  if constexpr (GEN && sizeof(R) == 4) return k_sweep<R, SH, BATCH, true>;
  else return k_sweep<R, SH, BATCH, false>;
}

// fn(std::integral_constant<int, shape>) for a sweep shape 0..kSweepShapes-1
template <class F>
static void with_shape(int shape, F&& fn) {
  switch (shape) {
    case 1: fn(std::integral_constant<int, 1>{}); break;
    case 2: fn(std::integral_constant<int, 2>{}); break;
    case 3: fn(std::integral_constant<int, 3>{}); break;
    case 4: fn(std::integral_constant<int, 4>{}); break;
    default: fn(std::integral_constant<int, 0>{}); break;
  }
}

// Grid of the sweep (every CTA gets at least one chunk).
static int sweep_grid(int grid, int nchunks) { return grid < nchunks ? grid : (nchunks > 0 ? nchunks : 1); }

template <class R>
static void launch_sweep(const DevFault<R>& f, int m_dt, int grid, int shape, cudaStream_t st) {
  if (f.nchunks == 0) return;
  const int gr = sweep_grid(grid, f.nchunks);
  const bool gen = sizeof(R) == 4 && f.gen_ds_max > 0.0f && f.wtab;
  with_shape(shape, [&](auto sh) {
    constexpr int SH = decltype(sh)::value;
    if (gen)
      sweep_kernel<R, SH, false, true>()<<<gr, sweep_threads(sizeof(R) == 4), sweep_smem<R, SH>(), st>>>(
          f, nullptr, f.chunks, f.nchunks, f.partial, m_dt, f.wtab, f.wtab_pieces, f.gen_ds_max, false);
    else
      k_sweep<R, SH, false, false><<<gr, kSweepThreads, sweep_smem<R, SH>(), st>>>(
          f, nullptr, f.chunks, f.nchunks, f.partial, m_dt, nullptr, 0, 0.0f, false);
  });
}

// The per-mode finish starts early behind the sweep (its blocks wait for
// the sweep's completion on the device instead of a launch after it).
template <class R>
static void launch_finish(const DevFault<R>& f, double2* outT, double2* outN, bool f32, int grid, cudaStream_t st) {
  const DevFault<R> fv = f;
  const int G = sweep_grid(grid, f.nchunks);
  launch_early(k_sweep_finish<R>, dim3((f.nmodes + 255) / 256), dim3(256), 0, st, fv, outT, outN, f32, G);
}

template <class R>
void launch_history(const DevFault<R>& f, int m_dt, int grid, cudaStream_t st, cudaEvent_t sweep_done) {
  launch_sweep<R>(f, m_dt, grid, f.sweep_shape, st);
  if (sweep_done) cudaEventRecord(sweep_done, st);
  launch_finish<R>(f, f.AT, f.AN, true, grid, st);
}

template <class R>
void launch_history_ahead(const DevFault<R>& f, int m_dt, int grid, cudaStream_t st) {
  // into BT/BN; the commit adds the new slot's term
  launch_sweep<R>(f, 2 * m_dt, grid, f.lag_shape, st);
  launch_finish<R>(f, f.BT, f.BN, false, grid, st);
}

template <class R>
int sweep_blocks_per_sm(int shape, bool gen) {
  int n = 0;
  with_shape(shape, [&](auto sh) {
    constexpr int SH = decltype(sh)::value;
    if (gen && sizeof(R) == 4)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<R, SH, false, true>(),
                                                    sweep_threads(true), sweep_smem<R, SH>());
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<R, SH, false, false>, kSweepThreads,
                                                    sweep_smem<R, SH>());
  });
  return n;
}

int sweep_chunk_slots(int precision, int shape) {
  int n = 0;
  with_shape(shape, [&](auto sh) {
    constexpr int SH = decltype(sh)::value;
    n = precision == 1 ? SweepCfg<float, SH>::kSlots : SweepCfg<double, SH>::kSlots;
  });
  return n;
}

template <class R>
void launch_history_persist(const DevFault<R>* fs, const Chunk* chunks, int nchunks, double4* partial,
                            const int2* mm, int TM, const int2* fc, int shape, int grid, int m_dt,
                            cudaStream_t st, bool ahead, const float4* wtab, int wtab_pieces, float gen_ds_max,
                            unsigned* bar_count, unsigned* bar_epoch, long long bar_limit, int members,
                            bool ring_evict_first) {
  const bool gen = sizeof(R) == 4 && wtab && gen_ds_max > 0.0f;
  const SweepBarrier bar{bar_count, bar_epoch, bar_limit, members};
  with_shape(shape, [&](auto sh) {
    constexpr int SH = decltype(sh)::value;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.dynamicSmemBytes = sweep_smem<R, SH>();
    if (gen) {
      if constexpr (sizeof(R) == 4) {
        cfg.blockDim = dim3(sweep_threads(true));
        cudaLaunchKernelEx(&cfg, k_sweep_persist<R, SH, true>, fs, chunks, nchunks, partial, m_dt, wtab, wtab_pieces,
                           gen_ds_max, mm, TM, fc, ahead, bar, ring_evict_first);
      }
    } else {
      cfg.blockDim = dim3(sweep_threads(false));
      cudaLaunchKernelEx(&cfg, k_sweep_persist<R, SH, false>, fs, chunks, nchunks, partial, m_dt,
                         static_cast<const float4*>(nullptr), 0, 0.0f, mm, TM, fc, ahead, bar, ring_evict_first);
    }
  });
}

// Resident CTAs per SM of the persistent ensemble sweep (its cooperative
// grid must fit at once).
template <class R>
int persist_blocks_per_sm(int shape, bool gen) {
  int n = 0;
  with_shape(shape, [&](auto sh) {
    constexpr int SH = decltype(sh)::value;
    if (gen && sizeof(R) == 4)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_persist<R, SH, sizeof(R) == 4>, sweep_threads(true),
                                                    sweep_smem<R, SH>());
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_persist<R, SH, false>, sweep_threads(false),
                                                    sweep_smem<R, SH>());
  });
  return n;
}

template <class R>
void launch_history_batch(const DevFault<R>* fs, const Chunk* chunks, int nchunks, double4* partial,
                          const int2* mm, int TM, const int2* fc, int shape, int grid, int m_dt,
                          cudaStream_t st, bool ahead, const float4* wtab, int wtab_pieces, float gen_ds_max,
                          bool ring_evict_first) {
  const int G = sweep_grid(grid, nchunks);
  if (nchunks > 0)
    with_shape(shape, [&](auto sh) {
      constexpr int SH = decltype(sh)::value;
      DevFault<R> none{};
      if (sizeof(R) == 4 && wtab && gen_ds_max > 0.0f)
        sweep_kernel<R, SH, true, true>()<<<G, sweep_threads(sizeof(R) == 4), sweep_smem<R, SH>(), st>>>(
            none, fs, chunks, nchunks, partial, m_dt, wtab, wtab_pieces, gen_ds_max, ring_evict_first);
      else
        k_sweep<R, SH, true, false><<<G, kSweepThreads, sweep_smem<R, SH>(), st>>>(
            none, fs, chunks, nchunks, partial, m_dt, nullptr, 0, 0.0f, ring_evict_first);
    });
  k_sweep_finish_b<R><<<(TM + 255) / 256, 256, 0, st>>>(fs, mm, TM, fc, nchunks, G, partial, ahead);
}

template <class R>
void launch_pass_batch(const FftGeom& g, const DevFault<R>* fs, int members, int N, int pass, int m_dt,
                       cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {
    if (N <= kFusedMaxN) {
      with_lgn(N, [&](auto lg) {
        constexpr int LG = decltype(lg)::value;
        if constexpr ((1 << LG) >= kClusterMinN) {
          launch_cluster_kernel(k_spectral_cluster_b<LG, kClusterEPT>, members, N, batch_cluster_ctas(N), st, false,
                                static_cast<cudaEvent_t>(nullptr), fs, pass, m_dt);
        } else {
          k_spectral_fused_b<LG><<<members, N / 8, fused_smem(N), st>>>(fs, pass, m_dt);
        }
      });
      k_newton_b<R><<<dim3((N + 31) / 32, members), 32, 0, st>>>(fs, pass, m_dt);
      return;
    }
  }
  const size_t cs = col_smem<R>(g), rs = row_smem<R>(g);
  const dim3 gc(g.N1 / g.Bc, members), gr(g.N2 / g.Br, members);
  k_col_b<R, false, PRO_PASS><<<gc, g.tc, cs, st>>>(g, fs, pass, m_dt);
  k_row_b<R, false><<<gr, g.tr, rs, st>>>(g, fs);
  k_col_b<R, true, PRO_ASSEMBLE><<<gc, g.tc, cs, st>>>(g, fs, pass, m_dt);
  k_row_b<R, true><<<gr, g.tr, rs, st>>>(g, fs);
  k_newton_b<R><<<dim3((N + 31) / 32, members), 32, 0, st>>>(fs, pass, m_dt);  // members use 32 per warp
}

template <class R>
void launch_commit_batch(const DevFault<R>* fs, int members, int N, int m_dt, cudaStream_t st, int lag_p) {
  const int n = N;  // N > N/2 + 1 modes
  k_commit_b<R><<<dim3((n + 255) / 256, members), 256, 0, st>>>(fs, m_dt, lag_p);
}

template <class R>
void configure_batch_kernels(const FftGeom& g) {
  if constexpr (sizeof(R) == 4) {
    if (g.N <= kFusedMaxN)
      with_lgn(g.N, [&](auto lg) {
        constexpr int LG = decltype(lg)::value;
        if constexpr ((1 << LG) >= kClusterMinN) {
          allow_smem(k_spectral_cluster_b<LG, kClusterEPT>, cluster_smem(g.N, batch_cluster_ctas(g.N)));
          cudaFuncSetAttribute(k_spectral_cluster_b<LG, kClusterEPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        } else {
          allow_smem(k_spectral_fused_b<LG>, fused_smem(g.N));
        }
      });
  }
  allow_smem(k_col_b<R, false, PRO_PASS>, col_smem<R>(g));
  allow_smem(k_col_b<R, true, PRO_ASSEMBLE>, col_smem<R>(g));
  allow_smem(k_row_b<R, false>, row_smem<R>(g));
  allow_smem(k_row_b<R, true>, row_smem<R>(g));
}

template <class R>
int history_blocks_per_sm() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_history_t<R, false>, kHistThreads, 0);
  return n;
}

template <class R>
void launch_push_multi(const DevFault<R>& f, int m_dt, cudaStream_t st) {
  if (f.nchunks == 0) return;
  const int grid = f.nchunks < 4096 ? f.nchunks : 4096;
  k_push_multi<R><<<grid, 256, 0, st>>>(f, m_dt);
}

template <class R>
void launch_weight_pow2(const DevFault<R>& f, cudaStream_t st) {
  k_weight_pow2<R><<<f.nmodes, 256, 0, st>>>(f.w, f.w_off, f.Mn, f.nmodes, f.w0pow, f.c0pow, f.S, f.mu, f.dt_min);
}

template <class R>
void launch_ring_undo(const DevFault<R>& f, int m_dt, void* undo, int dir, cudaStream_t st) {
  if (f.nchunks == 0) return;
  const int grid = f.nchunks < 4096 ? f.nchunks : 4096;
  k_ring_undo<R><<<grid, 256, 0, st>>>(f, m_dt, static_cast<Slot<R>*>(undo), dir);
}

// Plain streaming read of n16 float4s (grid-stride, eight loads in flight
// per thread): see sbiem_read_probe.
__global__ void __launch_bounds__(256) k_read_probe(const float4* __restrict__ p, int64_t n16, float* sink) {
  constexpr int U = 8;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  float acc = 0.f;
  for (; i + (U - 1) * stride < n16; i += U * stride) {
    float4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = __ldcs(p + i + u * stride);
#pragma unroll
    for (int u = 0; u < U; ++u) acc += (v[u].x + v[u].y) + (v[u].z + v[u].w);
  }
  for (; i < n16; i += stride) {
    const float4 v = __ldcs(p + i);
    acc += (v.x + v.y) + (v.z + v.w);
  }
  if (acc == -1234.5f) *sink = acc;
}

void launch_read_probe(const void* p, int64_t bytes, float* sink, int sm_count, cudaStream_t st) {
  k_read_probe<<<4 * sm_count, 256, 0, st>>>(static_cast<const float4*>(p), bytes / 16, sink);
}

__global__ void k_to_float2(const double2* a, float2* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2(static_cast<float>(a[i].x), static_cast<float>(a[i].y));
}

void launch_to_float2(const double2* a, float2* out, int n, cudaStream_t st) {
  k_to_float2<<<(n + 255) / 256, 256, 0, st>>>(a, out, n);
}

// Ring slots from two device arrays of interleaved complex values (shear,
// normal), FP64 (in_f32 = false) or FP32, converted to the ring's precision.
template <class R, class I>
__global__ void k_set_ring(Slot<R>* ring, const I* __restrict__ hT, const I* __restrict__ hN, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    Slot<R> v;
    if constexpr (sizeof(R) == 4) {
      v = make_float4(static_cast<float>(hT[2 * i]), static_cast<float>(hT[2 * i + 1]),
                      static_cast<float>(hN[2 * i]), static_cast<float>(hN[2 * i + 1]));
    } else {
      v.t = make_double2(static_cast<double>(hT[2 * i]), static_cast<double>(hT[2 * i + 1]));
      v.n = make_double2(static_cast<double>(hN[2 * i]), static_cast<double>(hN[2 * i + 1]));
    }
    ring[i] = v;
  }
}

template <class R>
void launch_set_ring(Slot<R>* ring, const void* hT, const void* hN, bool in_f32, int64_t n, int sm_count,
                     cudaStream_t st) {
  if (n <= 0) return;
  const int grid = 4 * sm_count;
  if (in_f32)
    k_set_ring<R, float><<<grid, 256, 0, st>>>(ring, static_cast<const float*>(hT), static_cast<const float*>(hN), n);
  else
    k_set_ring<R, double><<<grid, 256, 0, st>>>(ring, static_cast<const double*>(hT), static_cast<const double*>(hN),
                                                n);
}
template void launch_set_ring<float>(Slot<float>*, const void*, const void*, bool, int64_t, int, cudaStream_t);
template void launch_set_ring<double>(Slot<double>*, const void*, const void*, bool, int64_t, int, cudaStream_t);

__global__ void k_zin(const double* V, const double* kappa, float2* zin, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) zin[i] = make_float2(static_cast<float>(V[i]), static_cast<float>(kappa[i] * V[i]));
}

void launch_zin(const double* V, const double* kappa, float2* zin, int n, cudaStream_t st) {
  k_zin<<<(n + 255) / 256, 256, 0, st>>>(V, kappa, zin, n);
}

void launch_maxdiff(const double* a, const double* b, int n, double* out, cudaStream_t st) {
  k_maxdiff<<<1, 1024, 0, st>>>(a, b, n, out);
}

template <class R>
void launch_commit(const DevFault<R>& f, int m_dt, cudaStream_t st, int lag_p) {
  const int n = f.N > f.nmodes ? f.N : f.nmodes;
  const int nt = 256;
  launch_early(k_commit<R>, dim3((n + nt - 1) / nt), dim3(nt), 0, st, f, m_dt, m_dt * f.dt_min, lag_p);
}

template <class R>
void launch_weights(const DevFault<R>& f, const double* cheb, int npieces, int deg, double h, double cs,
                    const int32_t* MT, const int32_t* MN, int quadrature, cudaStream_t st) {
  k_weights<R><<<f.nmodes, 256, 0, st>>>(f.w, f.w_off, f.Mn, f.nmodes, f.L, cs, f.dt_min, cheb, npieces, deg, h,
                                         MT, MN, quadrature);
}

void launch_fft64(const FftGeom& g, const double2* tw, const double2* in, double2* tmp, double2* out,
                  bool inverse, cudaStream_t st) {
  DevFault<double> none{};
  const size_t cs = col_smem<double>(g), rs = row_smem<double>(g);
  if (!inverse) {
    auto kc = k_col<double, false, PRO_LOAD>;
    auto kr = k_row<double, false>;
    kc<<<g.N1 / g.Bc, g.tc, cs, st>>>(g, tw, in, tmp, none, 0, 0, 0.0);
    kr<<<g.N2 / g.Br, g.tr, rs, st>>>(g, tw, tmp, out, 1.0, nullptr);
  } else {
    auto kc = k_col<double, true, PRO_LOAD>;
    auto kr = k_row<double, true>;
    kc<<<g.N1 / g.Bc, g.tc, cs, st>>>(g, tw, in, tmp, none, 0, 0, 0.0);
    kr<<<g.N2 / g.Br, g.tr, rs, st>>>(g, tw, tmp, out, 1.0 / g.N, nullptr);
  }
}

void launch_pack(int N, const double* x, const double* y, const double* ymul, double2* z, cudaStream_t st) {
  k_pack<<<(N + 255) / 256, 256, 0, st>>>(N, x, y, ymul, z);
}
void launch_unpack(int N, const double2* Z, double2* X, double2* Y, cudaStream_t st) {
  k_unpack<<<(N / 2 + 1 + 255) / 256, 256, 0, st>>>(N, Z, X, Y);
}
void launch_d2(int N, double L, double2* Z, cudaStream_t st) { k_d2<<<(N + 255) / 256, 256, 0, st>>>(N, L, Z); }
void launch_real_part(int N, const double2* z, double* x, cudaStream_t st) {
  k_real_part<<<(N + 255) / 256, 256, 0, st>>>(N, z, x);
}

template <class R>
void configure_kernels(const FftGeom& g) {
  for (int sh = 0; sh < kSweepShapes; ++sh)
    with_shape(sh, [&](auto shc) {
      constexpr int SH = decltype(shc)::value;
      allow_smem(k_sweep<R, SH, false, false>, sweep_smem<R, SH>());
      allow_smem(k_sweep<R, SH, true, false>, sweep_smem<R, SH>());
      allow_smem(k_sweep_persist<R, SH, false>, sweep_smem<R, SH>());
      if constexpr (sizeof(R) == 4) {
        allow_smem(k_sweep<R, SH, false, true>, sweep_smem<R, SH>());
        allow_smem(k_sweep<R, SH, true, true>, sweep_smem<R, SH>());
        allow_smem(k_sweep_persist<R, SH, true>, sweep_smem<R, SH>());
      }
    });
  if constexpr (sizeof(R) == 4) {
    if (g.N <= kFusedMaxN)
      with_lgn(g.N, [&](auto lg) {
        constexpr int LG = decltype(lg)::value;
        if constexpr ((1 << LG) >= kClusterMinN) {
          allow_smem(k_spectral_cluster<LG, kClusterEPT>, cluster_smem(g.N, cluster_ctas(g.N)));
          cudaFuncSetAttribute(k_spectral_cluster<LG, kClusterEPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        } else {
          allow_smem(k_spectral_fused<LG>, fused_smem(g.N));
        }
      });
  }
  const size_t cs = col_smem<R>(g), rs = row_smem<R>(g);
  allow_smem(k_col<R, false, PRO_PASS>, cs);
  allow_smem(k_col<R, true, PRO_ASSEMBLE>, cs);
  allow_smem(k_row<R, false>, rs);
  allow_smem(k_row<R, true>, rs);
  const FftGeom g64 = make_geom(g.N, sizeof(double2));
  allow_smem(k_col<double, false, PRO_LOAD>, col_smem<double>(g64));
  allow_smem(k_col<double, true, PRO_LOAD>, col_smem<double>(g64));
  allow_smem(k_row<double, false>, row_smem<double>(g64));
  allow_smem(k_row<double, true>, row_smem<double>(g64));
}

template void launch_history_persist<double>(const DevFault<double>*, const Chunk*, int, double4*, const int2*, int,
                                             const int2*, int, int, int, cudaStream_t, bool, const float4*, int,
                                             float, unsigned*, unsigned*, long long, int, bool);
template void launch_history_persist<float>(const DevFault<float>*, const Chunk*, int, double4*, const int2*, int,
                                            const int2*, int, int, int, cudaStream_t, bool, const float4*, int,
                                            float, unsigned*, unsigned*, long long, int, bool);
template int persist_blocks_per_sm<double>(int, bool);
template int persist_blocks_per_sm<float>(int, bool);
template void launch_history_batch<double>(const DevFault<double>*, const Chunk*, int, double4*, const int2*, int,
                                           const int2*, int, int, int, cudaStream_t, bool, const float4*, int,
                                           float, bool);
template void launch_history_batch<float>(const DevFault<float>*, const Chunk*, int, double4*, const int2*, int,
                                          const int2*, int, int, int, cudaStream_t, bool, const float4*, int,
                                          float, bool);
template void launch_pass_batch<double>(const FftGeom&, const DevFault<double>*, int, int, int, int, cudaStream_t);
template void launch_pass_batch<float>(const FftGeom&, const DevFault<float>*, int, int, int, int, cudaStream_t);
template void launch_commit_batch<double>(const DevFault<double>*, int, int, int, cudaStream_t, int);
template void launch_commit_batch<float>(const DevFault<float>*, int, int, int, cudaStream_t, int);
template void configure_batch_kernels<double>(const FftGeom&);
template void configure_batch_kernels<float>(const FftGeom&);
template int history_blocks_per_sm<double>();
template int history_blocks_per_sm<float>();
template void configure_kernels<double>(const FftGeom&);
template void configure_kernels<float>(const FftGeom&);
template void launch_history<double>(const DevFault<double>&, int, int, cudaStream_t, cudaEvent_t);
template void launch_history<float>(const DevFault<float>&, int, int, cudaStream_t, cudaEvent_t);
template void launch_pass<double>(const DevFault<double>&, int, int, cudaStream_t);
template void launch_pass<float>(const DevFault<float>&, int, int, cudaStream_t);
template void launch_spectral<double>(const DevFault<double>&, int, int, cudaStream_t, cudaEvent_t);
template void launch_spectral<float>(const DevFault<float>&, int, int, cudaStream_t, cudaEvent_t);
template void launch_newton<double>(const DevFault<double>&, int, int, cudaStream_t);
template void launch_newton<float>(const DevFault<float>&, int, int, cudaStream_t);
template void launch_push_multi<double>(const DevFault<double>&, int, cudaStream_t);
template void launch_push_multi<float>(const DevFault<float>&, int, cudaStream_t);
template void launch_weight_pow2<double>(const DevFault<double>&, cudaStream_t);
template void launch_weight_pow2<float>(const DevFault<float>&, cudaStream_t);
template void launch_ring_undo<double>(const DevFault<double>&, int, void*, int, cudaStream_t);
template void launch_ring_undo<float>(const DevFault<float>&, int, void*, int, cudaStream_t);
template void launch_commit<double>(const DevFault<double>&, int, cudaStream_t, int);
template void launch_commit<float>(const DevFault<float>&, int, cudaStream_t, int);
template void launch_history_ahead<double>(const DevFault<double>&, int, int, cudaStream_t);
template void launch_history_ahead<float>(const DevFault<float>&, int, int, cudaStream_t);
template void launch_history_atomic<double>(const DevFault<double>&, int, int, cudaStream_t);
template void launch_history_atomic<float>(const DevFault<float>&, int, int, cudaStream_t);
template int sweep_blocks_per_sm<double>(int, bool);
template int sweep_blocks_per_sm<float>(int, bool);
template void launch_weights<double>(const DevFault<double>&, const double*, int, int, double, double,
                                     const int32_t*, const int32_t*, int, cudaStream_t);
template void launch_weights<float>(const DevFault<float>&, const double*, int, int, double, double,
                                    const int32_t*, const int32_t*, int, cudaStream_t);

}  // namespace sbiem
