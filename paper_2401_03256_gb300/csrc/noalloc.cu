// noalloc.cu - Static PageRank over a caller's device CSR without any device allocation.
//
// The library's graph handles own their device memory (cudaMalloc at creation and on
// growth).  Some callers cannot allow that: code whose device memory all comes from a host
// application's own pool or budget, code on latency-critical paths where the implicit
// device-wide synchronisation of cudaMalloc / cudaFree would stall other streams, and
// plugins that are handed device buffers but no right to allocate.  pr_static_noalloc
// serves them: the caller passes the graph and the output ranks in device memory, and the
// only working memory is the fixed array below, a file-scope __device__ array that exists
// on every device that loads this library, from module load until the process exits.
//
// Host code never names that array as an address: in host code its name is a host-side
// stand-in.  The device address is fetched once per device with cudaGetSymbolAddress, with
// that device current, on the first call on the device, and passed to the kernels.
//
// Every call uses the same array, and a call leaves its contents behind: the control words
// and out-degree counters are cleared at the start of each call.  Calls whose work overlaps
// on the GPU (two host threads, or two streams of one device) race on the array.
#include <algorithm>
#include <mutex>

#include "prdf_common.cuh"
#include "../../include/prdf.h"

namespace {

constexpr uint32_t kMaxN = PR_NOALLOC_MAX_VERTICES;
constexpr int kThreads = 256;
constexpr int kChunkIters = 8;     // iteration launches between reads of the control block
constexpr int kMaxDevices = 64;

struct NaCtl {
  unsigned long long dmax;  // max |Delta R| of the running iteration (bits of a double >= 0)
  uint32_t arrived;         // blocks finished with the running iteration
  uint32_t done;            // 1 once an iteration's max change was <= tol
  uint32_t bad;             // 1 malformed offsets, 2 column id >= n, 4 vertex without out-edges
  int32_t iterations;
  double last_delta;
};

// Layout: control block (256 bytes), out-degrees [kMaxN], contributions c0 [kMaxN], c1 [kMaxN].
constexpr size_t kCtlBytes = 256;
constexpr size_t kDegBytes = sizeof(uint32_t) * kMaxN;
constexpr size_t kContribBytes = sizeof(double) * kMaxN;
constexpr size_t kScratchBytes = kCtlBytes + kDegBytes + 2 * kContribBytes;
static_assert(sizeof(NaCtl) <= kCtlBytes, "control block");
static_assert(kScratchBytes == PR_NOALLOC_SCRATCH_BYTES, "scratch size stated in prdf.h");

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_addr_mu;
unsigned char *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};  // multiprocessors of each device, read with the address

// off must be non-decreasing from 0 to m.
__global__ void k_na_offsets(const uint64_t *off, uint32_t n, uint64_t m, NaCtl *ctl) {
  uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v > n) return;
  bool ok = v == 0 ? off[0] == 0 : off[v - 1] <= off[v];
  if (v == n) ok = ok && off[n] == m;
  if (!ok) atomicOr(&ctl->bad, 1u);
}

// Out-degree of u = its appearances as a source in the in-edge rows.
__global__ void k_na_degree(const uint32_t *col, uint64_t m, uint32_t n, uint32_t *deg, NaCtl *ctl) {
  uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  uint32_t u = col[e];
  if (u >= n) atomicOr(&ctl->bad, 2u);
  else atomicAdd(&deg[u], 1u);
}

__global__ void k_na_check_deg(const uint32_t *deg, uint32_t n, NaCtl *ctl) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n && deg[v] == 0) atomicOr(&ctl->bad, 4u);
}

// R = 1/n, c = R / |out(u)|.
__global__ void k_na_init(uint32_t n, const uint32_t *deg, double *R, double *c) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double r = 1.0 / (double)n;
  R[v] = r;
  c[v] = r / (double)deg[v];
}

// One Jacobi iteration of Eq. 1: R[v] = (1 - alpha) / n + alpha * sum over in-edges (u, v)
// of c_in[u]; c_out[v] = R[v] / |out(v)|.  The rank is updated in place (the sums read only
// c_in).  The last block to finish folds the iteration's L-inf change into the control
// block and sets done once it is <= tol; launches after that return at once.
__global__ void __launch_bounds__(kThreads) k_na_iter(uint32_t n, const uint64_t *off, const uint32_t *col,
                                                      const uint32_t *deg, double base, double alpha, double tol,
                                                      const double *c_in, double *c_out, double *R, NaCtl *ctl,
                                                      int32_t it) {
  __shared__ double s_max[kThreads / 32];
  if (*(volatile uint32_t *)&ctl->done) return;
  double lmax = 0.0;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (uint64_t e = off[v], end = off[v + 1]; e < end; e++) s += c_in[col[e]];
    const double r = base + alpha * s;
    lmax = fmax(lmax, fabs(r - R[v]));
    R[v] = r;
    c_out[v] = r / (double)deg[v];
  }
  for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = lmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bmax = s_max[0];
    for (int w = 1; w < kThreads / 32; w++) bmax = fmax(bmax, s_max[w]);
    atomicMax(&ctl->dmax, (unsigned long long)__double_as_longlong(bmax));
    __threadfence();
    if (atomicAdd(&ctl->arrived, 1u) == gridDim.x - 1) {
      __threadfence();
      const double d = __longlong_as_double((long long)atomicAdd(&ctl->dmax, 0ull));
      ctl->last_delta = d;
      ctl->iterations = it + 1;
      if (d <= tol) ctl->done = 1;
      ctl->dmax = 0;
      ctl->arrived = 0;
    }
  }
}

bool on_device(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

inline unsigned blocks_for(uint64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

extern "C" pr_status pr_static_noalloc(uint32_t n, int64_t m, const uint64_t *in_off, const uint32_t *in_col,
                                       const pr_params *params, void *cuda_stream, double *ranks, pr_stats *stats) {
  if (stats) *stats = pr_stats{};
  if (n > kMaxN) return PR_ERR_CAPACITY;  // more vertices than the fixed scratch holds
  pr_params p;
  if (params) p = *params; else pr_params_default(&p);
  if (n == 0 || m < 0 || !in_off || !ranks || (m > 0 && !in_col)) return PR_ERR_INVALID_ARG;
  if (!(p.alpha > 0.0 && p.alpha < 1.0) || !(p.tol >= 0.0) || p.max_iter < 0 || p.max_iter > prdf::kMaxIterLimit ||
      p.precision != PR_F64 || p.dead_end != PR_DEADEND_SELFLOOP)
    return PR_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return PR_ERR_CUDA;
  }
  if (!on_device(in_off, dev) || !on_device(ranks, dev) || (m > 0 && !on_device(in_col, dev)))
    return PR_ERR_INVALID_ARG;
  unsigned char *base_ptr = nullptr;
  int sm_count = 0;
  {
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
      void *a = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
      if (e != cudaSuccess || !a) {
        cudaGetLastError();
        return PR_ERR_CUDA;
      }
      int sms = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return PR_ERR_CUDA;
      }
      g_sms[dev] = sms;
      g_addr[dev] = (unsigned char *)a;
    }
    base_ptr = g_addr[dev];
    sm_count = g_sms[dev];
  }
  NaCtl *ctl = (NaCtl *)base_ptr;
  uint32_t *deg = (uint32_t *)(base_ptr + kCtlBytes);
  double *c[2] = {(double *)(base_ptr + kCtlBytes + kDegBytes),
                  (double *)(base_ptr + kCtlBytes + kDegBytes + kContribBytes)};
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // checks of the caller's CSR first: nothing is written to ranks unless it is well formed
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(NaCtl), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(deg, 0, sizeof(uint32_t) * n, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PR_ERR_CUDA;
  }
  k_na_offsets<<<blocks_for((uint64_t)n + 1), kThreads, 0, st>>>(in_off, n, (uint64_t)m, ctl);
  prdf::count_launch();
  if (m > 0) {
    k_na_degree<<<blocks_for((uint64_t)m), kThreads, 0, st>>>(in_col, (uint64_t)m, n, deg, ctl);
    prdf::count_launch();
  }
  k_na_check_deg<<<blocks_for(n), kThreads, 0, st>>>(deg, n, ctl);
  prdf::count_launch();
  NaCtl h{};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl, sizeof(NaCtl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return PR_ERR_CUDA;
  if (h.bad & 2u) return PR_ERR_VERTEX_RANGE;
  if (h.bad) return PR_ERR_INVALID_ARG;  // malformed offsets, or a vertex without out-edges

  k_na_init<<<blocks_for(n), kThreads, 0, st>>>(n, deg, ranks, c[0]);
  prdf::count_launch();
  const double base = (1.0 - p.alpha) / (double)n;
  const unsigned grid = std::min<unsigned>(blocks_for(n), (unsigned)sm_count * 8u);  // grid-stride rows
  int32_t it = 0;
  while (it < p.max_iter) {
    const int32_t k = std::min<int32_t>(kChunkIters, p.max_iter - it);
    for (int32_t j = 0; j < k; j++, it++) {
      k_na_iter<<<grid, kThreads, 0, st>>>(n, in_off, in_col, deg, base, p.alpha, p.tol, c[it & 1],
                                           c[(it + 1) & 1], ranks, ctl, it);
      prdf::count_launch();
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl, sizeof(NaCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return PR_ERR_CUDA;
    if (h.done) break;
  }
  if (p.max_iter == 0) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return PR_ERR_CUDA;
  }
  if (stats) {
    stats->iterations = h.iterations;
    stats->converged = h.done ? 1 : 0;
    stats->affected_final = n;
    stats->vertices_processed = (int64_t)h.iterations * n;
    stats->edges_processed = (int64_t)h.iterations * m;
    stats->bytes_algorithmic = (double)h.iterations * (12.0 * (double)m + 36.0 * (double)n);
    stats->last_delta = h.last_delta;
  }
  return PR_OK;
}
