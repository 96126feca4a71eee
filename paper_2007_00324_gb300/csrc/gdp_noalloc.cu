// Bad-element scan for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running under an
// allocator that must not be re-entered (inside another library's memory
// callbacks), processes whose device memory is entirely pre-reserved by a
// framework pool, or hard real-time paths where an allocation could block.
// gdp_scan_noalloc gives them the scan of the refinement loop (per triangle:
// the radius-edge test and, per subsegment edge, the encroachment test by the
// triangle's own apex, with circumcentres / midpoints and priority measure
// bits) on a triangulation they hold in their own device buffers, writing into
// output buffers they own.  The only extra memory is the file-scope array
// below, which every GPU that loads this library keeps until the process
// exits.
#include <cuda_runtime.h>

#include <mutex>

#include "gdp.h"
#include "gdp_pred.cuh"

namespace {

constexpr int NA_BS = 256;
constexpr int NA_MAX_TRI = GDP_NOALLOC_MAX_TRIANGLES;   // 4 Mi triangles
constexpr int NA_GRID = 1024;                           // fixed launch width

struct NoallocScratch {
  unsigned char cnt[NA_MAX_TRI];   // entries each triangle contributes (0..4)
  int blk[NA_GRID];                // per-block entry counts
  int total;                       // entries found by the last call
  int err;                         // set when an index is out of range
};

// about 4.2 MB, shared by every call on the device
static __device__ __align__(256) NoallocScratch g_scratch;

__device__ __forceinline__ int na_comp(const int4& a, int i) {
  return i == 0 ? a.x : (i == 1 ? a.y : a.z);
}

__device__ __forceinline__ int na_entries(const double2* V, const int4& T4, int n_vert, double B2,
                                          int* err) {
  if (T4.x < 0 || T4.y < 0 || T4.z < 0 || T4.x >= n_vert || T4.y >= n_vert || T4.z >= n_vert) {
    atomicOr(err, 1);
    return 0;
  }
  const gdp::TriTerms tt = gdp::tri_terms(V[T4.x], V[T4.y], V[T4.z]);
  int c = gdp::is_bad(tt, B2) ? 1 : 0;
  for (int e = 0; e < 3; ++e) {
    if (!((T4.w >> e) & 1)) continue;
    const double2 u = V[na_comp(T4, (e + 1) % 3)], v = V[na_comp(T4, (e + 2) % 3)];
    if (gdp::dot_sign(u, v, V[na_comp(T4, e)]) < 0) ++c;
  }
  return c;
}

__device__ int na_block_sum(int v, int* sm) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  if (w == 0) {
    int r = l < (int)(blockDim.x >> 5) ? sm[l] : 0;
    for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (l == 0) sm[32] = r;
  }
  __syncthreads();
  const int r = sm[32];
  __syncthreads();
  return r;
}

__device__ int na_excl_scan(int v, int* sm, int& total) {
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (l >= o) x += y;
  }
  __syncthreads();
  if (l == 31) sm[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = l < nw ? sm[l] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (l >= o) s += y;
    }
    if (l < nw) sm[l] = s;
  }
  __syncthreads();
  const int base = w ? sm[w - 1] : 0;
  total = sm[nw - 1];
  __syncthreads();
  return base + x - v;
}

// pass 1: entries per triangle into scratch, per-block sums
__global__ void __launch_bounds__(NA_BS) k_na_count(const double2* V, const int4* T, int n_tri,
                                                    int n_vert, double B2, NoallocScratch* S) {
  __shared__ int sm[33];
  const int c = (n_tri + gridDim.x - 1) / gridDim.x;
  const int b0 = min(n_tri, (int)blockIdx.x * c), b1 = min(n_tri, b0 + c);
  int s = 0;
  for (int t = b0 + threadIdx.x; t < b1; t += NA_BS) {
    const int k = na_entries(V, T[t], n_vert, B2, &S->err);
    S->cnt[t] = (unsigned char)k;
    s += k;
  }
  s = na_block_sum(s, sm);
  if (threadIdx.x == 0) S->blk[blockIdx.x] = s;
}

// pass 2: stable write in triangle order (bad triangle first, then its edges)
__global__ void __launch_bounds__(NA_BS) k_na_write(const double2* V, const int4* T, int n_tri,
                                                    double B2, NoallocScratch* S, int* kind,
                                                    int* verts, double2* pt, unsigned* meas,
                                                    int cap) {
  __shared__ int sm[33];
  const int c = (n_tri + gridDim.x - 1) / gridDim.x;
  const int b0 = min(n_tri, (int)blockIdx.x * c), b1 = min(n_tri, b0 + c);
  int off = 0;
  for (int k = threadIdx.x; k < (int)blockIdx.x; k += NA_BS) off += S->blk[k];
  off = na_block_sum(off, sm);
  for (int base = b0; base < b1; base += NA_BS) {
    const int t = base + threadIdx.x;
    const int k = t < b1 ? S->cnt[t] : 0;
    int tot;
    int r = off + na_excl_scan(k, sm, tot);
    if (k) {
      const int4 T4 = T[t];
      const gdp::TriTerms tt = gdp::tri_terms(V[T4.x], V[T4.y], V[T4.z]);
      if (gdp::is_bad(tt, B2)) {
        if (r < cap) {
          kind[r] = 0;
          verts[3 * r] = T4.x; verts[3 * r + 1] = T4.y; verts[3 * r + 2] = T4.z;
          pt[r] = gdp::circumcenter(tt);
          meas[r] = gdp::measure_bits(fabs(tt.cr));
        }
        ++r;
      }
      for (int e = 0; e < 3; ++e) {
        if (!((T4.w >> e) & 1)) continue;
        const int u = na_comp(T4, (e + 1) % 3), v = na_comp(T4, (e + 2) % 3);
        if (gdp::dot_sign(V[u], V[v], V[na_comp(T4, e)]) < 0) {
          if (r < cap) {   // the midpoint: there is no segment data for shells here
            kind[r] = 1;
            verts[3 * r] = u; verts[3 * r + 1] = v; verts[3 * r + 2] = -1;
            pt[r] = gdp::midpoint(V[u], V[v]);
            meas[r] = gdp::measure_bits(gdp::seg_measure(V[u], V[v]));
          }
          ++r;
        }
      }
    }
    off += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) S->total = off;
}

// device address of the scratch array, looked up once per device (a reset of
// the device between calls is not supported: the cached address would be stale)
constexpr int NA_MAX_DEVICES = 64;
NoallocScratch* g_addr[NA_MAX_DEVICES] = {};
std::mutex g_addr_lock;

int scratch_for_current_device(NoallocScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return GDP_ERR_CUDA;
  }
  if (dev < 0 || dev >= NA_MAX_DEVICES) return GDP_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_addr_lock);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return GDP_ERR_CUDA;
    }
    g_addr[dev] = static_cast<NoallocScratch*>(p);
  }
  *out = g_addr[dev];
  return GDP_OK;
}

}  // namespace

extern "C" int gdp_scan_noalloc(const double* xy_device, int64_t n_vert, const int32_t* tri_device,
                                int64_t n_tri, double B, int32_t* kind_device,
                                int32_t* verts_device, double* pt_device, uint32_t* meas_device,
                                int64_t cap, int64_t* count, void* cuda_stream) {
  if (!xy_device || !tri_device || !count || n_vert <= 0 || n_tri < 0 || cap < 0 || !(B > 0))
    return GDP_ERR_INPUT;
  if (cap > 0 && (!kind_device || !verts_device || !pt_device || !meas_device)) return GDP_ERR_INPUT;
  if (n_tri > NA_MAX_TRI || n_vert > INT32_MAX || cap > INT32_MAX) return GDP_ERR_CAPACITY;
  if ((reinterpret_cast<uintptr_t>(tri_device) & 15) || (reinterpret_cast<uintptr_t>(xy_device) & 15))
    return GDP_ERR_INPUT;
  // the points are written as 16-byte (x, y) pairs
  if (cap > 0 && (reinterpret_cast<uintptr_t>(pt_device) & 15)) return GDP_ERR_INPUT;
  NoallocScratch* S = nullptr;
  const int st = scratch_for_current_device(&S);
  if (st != GDP_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  *count = 0;
  if (n_tri == 0) return GDP_OK;
  // the error flag accumulates with atomicOr: clear it (memset allocates nothing)
  if (cudaMemsetAsync(&S->err, 0, sizeof(int), s) != cudaSuccess) return GDP_ERR_CUDA;
  const double B2 = B * B;
  const double2* V = reinterpret_cast<const double2*>(xy_device);
  const int4* T = reinterpret_cast<const int4*>(tri_device);
  k_na_count<<<NA_GRID, NA_BS, 0, s>>>(V, T, (int)n_tri, (int)n_vert, B2, S);
  k_na_write<<<NA_GRID, NA_BS, 0, s>>>(V, T, (int)n_tri, B2, S, kind_device, verts_device,
                                       reinterpret_cast<double2*>(pt_device), meas_device, (int)cap);
  if (cudaGetLastError() != cudaSuccess) return GDP_ERR_CUDA;
  int host[2] = {0, 0};   // total, err
  if (cudaMemcpyAsync(&host[0], &S->total, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&host[1], &S->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GDP_ERR_CUDA;
  if (host[1]) return GDP_ERR_INPUT;
  *count = host[0];
  return GDP_OK;
}
