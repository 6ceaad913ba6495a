// sph_noalloc.cu -- cell-key sort that allocates nothing.
//
// Some callers cannot let a library allocate device memory: a host program
// that owns the whole device-memory budget (a plugin or co-simulation host
// that hands out fixed buffers), or a latency-sensitive loop where
// cudaMalloc/cudaFree, which may synchronise the device, is not acceptable.
// For them, sph_sort_cell_keys_static runs the same stable radix sort as the
// neighbour list, with its scratch space (key/index ping-pong buffers and
// digit histograms) in the fixed array below instead of allocated memory.
//
// The array is a file-scope __device__ variable, so every GPU that loads
// libsph.so holds it (4,457,472 bytes) until the process exits.  In host code
// its name is only a host-side stand-in, so its device address is looked up
// once per device with cudaGetSymbolAddress, with that device current.
#include <mutex>
#include <string>

#include "../../include/sph.h"
#include "sph_internal.cuh"

namespace {

constexpr int64_t kMaxKeys = SPH_SORT_STATIC_MAX_KEYS;
// exactly the scratch the sort needs for the largest accepted n
constexpr size_t kScratchBytes = sph::sort_temp_bytes(kMaxKeys);
static_assert(kScratchBytes >= sph::sort_temp_bytes(1), "scratch size");

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

int fail(int code, const std::string &msg) {
  sph::set_last_error(msg);  // read back with sph_last_error()
  return code;
}

}  // namespace

extern "C" int sph_sort_cell_keys_static(const uint32_t *keys_in, uint32_t *keys_out,
                                          uint32_t *perm_out, int64_t n, int32_t nbits,
                                          void *stream) {
  if (n < 0 || n > kMaxKeys) {
    return fail(SPH_ERR_ARG, "sph_sort_cell_keys_static: n = " + std::to_string(n) +
                                 " exceeds the static limit of " + std::to_string(kMaxKeys) +
                                 " keys");
  }
  if (nbits < 1 || nbits > 32) {
    return fail(SPH_ERR_ARG, "sph_sort_cell_keys_static: nbits must be in [1, 32]");
  }
  if (n == 0) return SPH_OK;
  if (!keys_in || !keys_out || !perm_out) {
    return fail(SPH_ERR_ARG, "sph_sort_cell_keys_static: null device pointer");
  }
  {
    // the passes ping-pong between the outputs and the scratch while other
    // blocks still read the input, so the three arrays must be disjoint
    const uintptr_t a = (uintptr_t)keys_in, b = (uintptr_t)keys_out, c = (uintptr_t)perm_out;
    const uintptr_t len = (uintptr_t)n * 4u;
    auto overlap = [len](uintptr_t x, uintptr_t y) { return x < y + len && y < x + len; };
    if (overlap(a, b) || overlap(a, c) || overlap(b, c)) {
      return fail(SPH_ERR_ARG, "sph_sort_cell_keys_static: keys_in, keys_out and perm_out "
                               "must not overlap");
    }
  }
  if (sph::radix_sort_temp_bytes(n) > kScratchBytes) {
    return fail(SPH_ERR_ARG, "sph_sort_cell_keys_static: scratch too small");
  }
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    return fail(SPH_ERR_CUDA, std::string("sph_sort_cell_keys_static: cudaGetDevice: ") +
                                  cudaGetErrorString(err));
  }
  void *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      // first call on this device: look up the array's device address
      void *p = nullptr;
      err = cudaGetSymbolAddress(&p, g_sort_scratch);
      if (err != cudaSuccess || !p) {
        return fail(SPH_ERR_CUDA, std::string("sph_sort_cell_keys_static: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(err));
      }
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  // Every scratch word the sort reads is written earlier in the same call
  // (histograms by the upsweep, totals by the digit scan), so the contents
  // left by a previous call need no clearing.
  sph::radix_sort(keys_in, keys_out, perm_out, (int)n, nbits, scratch, (cudaStream_t)stream);
  err = cudaGetLastError();
  if (err != cudaSuccess) {
    return fail(SPH_ERR_CUDA, std::string("sph_sort_cell_keys_static: launch: ") +
                                  cudaGetErrorString(err));
  }
  return SPH_OK;
}
