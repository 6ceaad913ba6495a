// sph_sort.cu -- stable LSD radix sort of 32-bit cell keys with their source
// index, for the neighbour list of Sect. 5.1, which orders the particles by
// the cell each one lies in.
//
// Each 8-bit pass is three launches:
//   upsweep      per-tile digit counts (warp-aggregated with match.any),
//   digit_scan   one block per digit: exclusive scan of that digit's counts
//                over the tiles, plus the digit total,
//   downsweep    per tile: stable ranks from warp match.any in index order,
//                then a scatter to digit base + tile offset + rank.
// Only ceil(nbits / 8) passes run.  No atomics touch global memory, so the
// output is deterministic.
#include "sph_internal.cuh"

namespace sph {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                  // per thread
constexpr int kTile = kThreads * kItems;   // 2048 keys per block
constexpr int kRadix = 256;
static_assert(kTile == kSortTile && kRadix == kSortRadix, "sort geometry");

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__global__ void __launch_bounds__(kThreads)
k_upsweep(const uint32_t *__restrict__ keys, int n, int shift, int ntiles,
          uint32_t *__restrict__ hist, const int *__restrict__ n_dev) {
  if (n_dev) n = min(n, *n_dev);  // the key count, when only the device knows it
  __shared__ uint32_t cnt[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += kThreads) cnt[d] = 0;
  __syncthreads();
  const int base = blockIdx.x * kTile;
  const int lane = threadIdx.x & 31;
  for (int r = 0; r < kItems; r++) {
    int i = base + r * kThreads + threadIdx.x;
    bool valid = i < n;
    unsigned act = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      uint32_t d = (keys[i] >> shift) & (kRadix - 1);
      unsigned peers = __match_any_sync(act, d);
      if ((peers & lanemask_lt()) == 0) atomicAdd(&cnt[d], __popc(peers));
    }
    (void)lane;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kThreads) hist[d * ntiles + blockIdx.x] = cnt[d];
}

// One block per digit: exclusive scan of hist[d][0..ntiles) in place.
__global__ void __launch_bounds__(1024)
k_digit_scan(uint32_t *__restrict__ hist, int ntiles, uint32_t *__restrict__ totals) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  uint32_t *row = hist + (size_t)blockIdx.x * ntiles;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < ntiles; base += 1024) {
    int i = base + threadIdx.x;
    uint32_t v = i < ntiles ? row[i] : 0;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t s = warp_sums[lane];
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;  // inclusive
    }
    __syncthreads();
    uint32_t excl = carry + (warp ? warp_sums[warp - 1] : 0) + x - v;
    if (i < ntiles) row[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kThreads)
k_downsweep(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
            uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int n,
            int shift, int ntiles, const uint32_t *__restrict__ hist,
            const uint32_t *__restrict__ totals,
            const int *__restrict__ n_dev) {
  if (n_dev) n = min(n, *n_dev);
  __shared__ uint32_t wcnt[kWarps][kRadix];
  __shared__ uint32_t gbase[kRadix];
  __shared__ uint32_t wsum[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += kThreads)
    for (int w = 0; w < kWarps; w++) wcnt[w][d] = 0;
  // digit base = exclusive scan of the digit totals (256 values, one per thread)
  {
    uint32_t v = totals[threadIdx.x];
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t off = 0;
    for (int w = 0; w < warp; w++) off += wsum[w];
    gbase[threadIdx.x] = off + x - v + hist[threadIdx.x * ntiles + blockIdx.x];
  }
  __syncthreads();

  const int base = blockIdx.x * kTile + warp * (kTile / kWarps);
  uint32_t k[kItems], v[kItems], loc[kItems];
  for (int r = 0; r < kItems; r++) {
    int i = base + r * 32 + lane;
    bool valid = i < n;
    unsigned act = __ballot_sync(0xffffffffu, valid);
    loc[r] = 0xffffffffu;
    if (valid) {
      k[r] = keys_in[i];
      v[r] = vals_in ? vals_in[i] : (uint32_t)i;
      uint32_t d = (k[r] >> shift) & (kRadix - 1);
      unsigned peers = __match_any_sync(act, d);
      uint32_t before = wcnt[warp][d];
      unsigned rank = __popc(peers & lanemask_lt());
      __syncwarp(act);
      if (rank == 0) wcnt[warp][d] = before + __popc(peers);
      __syncwarp(act);
      loc[r] = before + rank;
    }
  }
  __syncthreads();
  // per digit: exclusive prefix of the warp counts (warp order = index order)
  {
    int d = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < kWarps; w++) {
      uint32_t t = wcnt[w][d];
      wcnt[w][d] = run;
      run += t;
    }
  }
  __syncthreads();
  for (int r = 0; r < kItems; r++) {
    if (loc[r] == 0xffffffffu) continue;
    uint32_t d = (k[r] >> shift) & (kRadix - 1);
    uint32_t dst = gbase[d] + wcnt[warp][d] + loc[r];
    keys_out[dst] = k[r];
    vals_out[dst] = v[r];
  }
}

}  // namespace

size_t radix_sort_temp_bytes(int64_t n) { return sort_temp_bytes(n); }

void radix_sort(const uint32_t *keys_in, uint32_t *keys_out, uint32_t *perm_out, int n,
                int nbits, void *temp, cudaStream_t s, const int *n_dev) {
  if (n <= 0) return;
  int ntiles = (n + kTile - 1) / kTile;
  char *p = (char *)temp;
  uint32_t *ktmp = (uint32_t *)p;
  p += ((size_t)n * 4 + 255) / 256 * 256;
  uint32_t *vtmp = (uint32_t *)p;
  p += ((size_t)n * 4 + 255) / 256 * 256;
  uint32_t *hist = (uint32_t *)p;
  p += ((size_t)ntiles * kRadix * 4 + 255) / 256 * 256;
  uint32_t *totals = (uint32_t *)p;

  int passes = (nbits + 7) / 8;
  if (passes < 1) passes = 1;
  const uint32_t *kin = keys_in;
  const uint32_t *vin = nullptr;  // first pass: identity permutation
  for (int pass = 0; pass < passes; pass++) {
    // the last pass must land in keys_out/perm_out
    bool to_out = ((passes - 1 - pass) % 2) == 0;
    uint32_t *kout = to_out ? keys_out : ktmp;
    uint32_t *vout = to_out ? perm_out : vtmp;
    int shift = pass * 8;
    k_upsweep<<<ntiles, kThreads, 0, s>>>(kin, n, shift, ntiles, hist, n_dev);
    k_digit_scan<<<kRadix, 1024, 0, s>>>(hist, ntiles, totals);
    k_downsweep<<<ntiles, kThreads, 0, s>>>(kin, vin, kout, vout, n, shift, ntiles, hist,
                                            totals, n_dev);
    kin = kout;
    vin = vout;
  }
}

}  // namespace sph
