// History convolution without device allocation: the sums of
// sbiem_history_sums (Sec. 3.1 window, Sec. 3.3 step (2), midpoint weights)
// on caller-owned device buffers.  It runs the library's warp-per-chunk
// kernel (k_history_t: chunks handed out by an atomic counter, a mode's
// chunk sums added in chunk order by the warp that finishes last), not the
// handle's bulk-async sweep, whose static partition and per-mode finish
// need tables sized per fault.  Its scratch -- chunk table, per-chunk
// partial sums, per-mode counters -- is one fixed static device array
// instead of memory allocated by the library.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "kernels.cuh"
#include "sbiem.h"

using namespace sbiem;

namespace {

constexpr int kMaxModes = SBIEM_NOALLOC_MAX_MODES;
constexpr int kMaxChunks = SBIEM_NOALLOC_MAX_CHUNKS;
constexpr int kChunkSlots = 2048;
constexpr int kMaxDevices = 64;

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffHeader = 0;                                    // Header
constexpr size_t kOffChunks = 256;                                  // Chunk[kMaxChunks]
constexpr size_t kOffPartial = kOffChunks + align256(sizeof(Chunk) * kMaxChunks);   // double4[kMaxChunks]
constexpr size_t kOffCounter = kOffPartial + align256(sizeof(double4) * kMaxChunks);  // int[kMaxModes]
constexpr size_t kScratchBytes = kOffCounter + align256(sizeof(int) * kMaxModes);

struct Header {
  int nchunks;
  int overflow;
  int work;
  unsigned status;
};

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

unsigned char* g_addr[kMaxDevices];  // device address of g_scratch, per device

// One CTA: chunk counts per mode, exclusive scan over modes, chunk table,
// counters and the work counter cleared.  Sets overflow instead of writing
// past the table.
__global__ void k_noalloc_chunks(const int32_t* __restrict__ R, int nmodes, unsigned char* scratch) {
  Header* hd = reinterpret_cast<Header*>(scratch + kOffHeader);
  Chunk* chunks = reinterpret_cast<Chunk*>(scratch + kOffChunks);
  int* counter = reinterpret_cast<int*>(scratch + kOffCounter);
  __shared__ long long part[1024];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int per = (nmodes + nth - 1) / nth;
  const int m0 = tid * per, m1 = min(nmodes, m0 + per);
  long long cnt = 0;
  for (int n = m0; n < m1; ++n) {
    counter[n] = 0;
    cnt += (static_cast<long long>(R[n]) + kChunkSlots - 1) / kChunkSlots;
  }
  part[tid] = cnt;
  __syncthreads();
  if (tid == 0) {
    long long run = 0;
    for (int t = 0; t < nth; ++t) {
      const long long c = part[t];
      part[t] = run;
      run += c;
    }
    hd->nchunks = static_cast<int>(run > kMaxChunks ? 0 : run);
    hd->overflow = run > kMaxChunks ? 1 : 0;
    hd->work = 0;
    hd->status = 0u;
  }
  __syncthreads();
  if (hd->overflow) return;
  long long c = part[tid];
  for (int n = m0; n < m1; ++n) {
    const long long r = R[n];
    const int k = static_cast<int>((r + kChunkSlots - 1) / kChunkSlots);
    for (int q = 0; q < k; ++q) {
      Chunk ch;
      ch.mode = n;
      ch.first = static_cast<int32_t>(c - q);
      ch.count = k;
      ch.pad = 0;
      ch.i0 = static_cast<int64_t>(q) * kChunkSlots;
      ch.i1 = min(static_cast<long long>(q + 1) * kChunkSlots, r);
      chunks[c] = ch;
      ++c;
    }
  }
}

int setup(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SBIEM_ERR_CUDA;
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return SBIEM_ERR_CUDA;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return SBIEM_OK;
}

template <class R>
int run(int nmodes, int m, const void* ring, const void* weights, const int64_t* ring_off,
        const int64_t* w_off, const int32_t* Rn, const int32_t* Mn, const int32_t* head, double* AT,
        double* AN, cudaStream_t st) {
  unsigned char* scr = nullptr;
  int rc = setup(&scr);
  if (rc) return rc;
  k_noalloc_chunks<<<1, 1024, 0, st>>>(Rn, nmodes, scr);
  if (cudaGetLastError() != cudaSuccess) return SBIEM_ERR_CUDA;
  Header hd;
  if (cudaMemcpyAsync(&hd, scr + kOffHeader, sizeof(hd), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SBIEM_ERR_CUDA;
  if (hd.overflow) return SBIEM_ERR_INVALID;
  // AT / AN of modes without history are zero
  if (cudaMemsetAsync(AT, 0, sizeof(double2) * nmodes, st) != cudaSuccess ||
      cudaMemsetAsync(AN, 0, sizeof(double2) * nmodes, st) != cudaSuccess)
    return SBIEM_ERR_CUDA;
  DevFault<R> f{};
  f.nmodes = nmodes;
  f.ring = static_cast<Slot<R>*>(const_cast<void*>(ring));
  f.w = static_cast<W2<R>*>(const_cast<void*>(weights));
  f.ring_off = ring_off;
  f.w_off = w_off;
  f.Rn = Rn;
  f.Mn = Mn;
  f.head = const_cast<int32_t*>(head);
  f.AT = reinterpret_cast<double2*>(AT);
  f.AN = reinterpret_cast<double2*>(AN);
  Header* dh = reinterpret_cast<Header*>(scr + kOffHeader);
  f.chunks = reinterpret_cast<const Chunk*>(scr + kOffChunks);
  f.partial = reinterpret_cast<double4*>(scr + kOffPartial);
  f.counter = reinterpret_cast<int*>(scr + kOffCounter);
  f.work = &dh->work;
  f.status = &dh->status;
  f.nchunks = hd.nchunks;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = history_blocks_per_sm<R>();
  launch_history_atomic<R>(f, m, sms * (per_sm > 0 ? per_sm : 1), st);
  return cudaGetLastError() == cudaSuccess ? SBIEM_OK : SBIEM_ERR_CUDA;
}

}  // namespace

extern "C" int sbiem_history_sums_noalloc(int64_t nmodes, int32_t precision, int64_t m, const void* ring,
                                          const void* weights, const int64_t* ring_off, const int64_t* w_off,
                                          const int32_t* R, const int32_t* M, const int32_t* head, double* AT,
                                          double* AN, void* stream) {
  if (nmodes < 1 || nmodes > kMaxModes || m < 1 || m > (int64_t(1) << 30) ||
      (precision != 0 && precision != 1) || !ring || !weights || !ring_off || !w_off || !R || !M || !head ||
      !AT || !AN)
    return SBIEM_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == 1)
    return run<float>(static_cast<int>(nmodes), static_cast<int>(m), ring, weights, ring_off, w_off, R, M, head,
                      AT, AN, st);
  return run<double>(static_cast<int>(nmodes), static_cast<int>(m), ring, weights, ring_off, w_off, R, M, head,
                     AT, AN, st);
}
