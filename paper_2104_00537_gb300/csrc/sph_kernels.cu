// sph_kernels.cu -- the per-step kernels of the WCSPH hot path (DualSPHysics
// paper, arXiv 2104.00537) for sm_103a:
//   k_upload      host particles -> (cell, float offset) state + keys
//   k_reorder     gather the state into cell order, Tait pressure (Eq 28)
//   k_mark + k_fill_*   cell start table of the sorted order (Sect. 5.1)
//   k_interact    Wendland C2 pair loop: momentum with artificial viscosity
//                 (Eq 21-22), continuity with density diffusion (Eq 15,
//                 17-18), dynamic boundaries (Eq 36), Eq 35 reductions
//   k_dt          time step (Eq 35) and imposed-motion increments (Eq 37)
//   k_predictor   Symplectic half step (Eq 33-34)
//   k_corrector   Symplectic full step (Eq 33-34)
//   k_end_step    t += dt in FP64
//   k_export / k_diag / k_pair_stats   read-out and parity helpers
#include <algorithm>
#include <cfloat>

#include "sph_internal.cuh"
#include "sph_kernels.cuh"

namespace sph {

// ---- small helpers ----------------------------------------------------------

__device__ __forceinline__ float tait_pressure(const CaseConst &C, float rho) {
  // P = B ((rho/rho0)^gamma - 1), evaluated as B expm1(gamma log1p(e)) with
  // e = (rho - rho0)/rho0 so that no digits cancel near rho0.
  float e = (rho - C.rho0) * C.inv_rho0;
  return C.btait * expm1f(C.gamma * log1pf(e));
}

__device__ __forceinline__ void decode_cell(uint32_t lin, int nx, int ny, int &cx, int &cy,
                                            int &cz) {
  int t = (int)(lin / (uint32_t)nx);
  cx = (int)lin - t * nx;
  cz = t / ny;
  cy = t - cz * ny;
}

__device__ __forceinline__ float below(float cs) {  // largest float < cs
  return __int_as_float(__float_as_int(cs) - 1);
}

// New offset after adding disp (FP64) to a float offset in [0, cs); returns
// the cell shift.  The sum is formed in FP64; when its float rounding stays
// inside the cell (the common case) that rounding is the new offset, and
// only a particle that changes cell takes the FP64 floor / shift path.
__device__ __forceinline__ int shift_axis(float off, double disp, const CaseConst &C,
                                          float &off_out) {
  double x = (double)off + disp;
  const float xf = (float)x;
  if (xf >= 0.f && xf < C.csf) {
    off_out = xf;
    return 0;
  }
  double k = floor(x * C.inv_cs);
  x = fma(-k, C.cs, x);
  if (x < 0.0) {
    x += C.cs;
    k -= 1.0;
  } else if (x >= C.cs) {
    x -= C.cs;
    k += 1.0;
  }
  float f = (float)x;
  if (f >= C.csf) f = below(C.csf);
  if (f < 0.f) f = 0.f;
  off_out = f;
  return (int)k;
}

// ---- upload ------------------------------------------------------------------

__global__ void k_upload(int n, const double *__restrict__ pos, const float *__restrict__ vel,
                         const float *__restrict__ rho, const uint8_t *__restrict__ type,
                         const int32_t *__restrict__ group, int slot, uint32_t id_base,
                         const CaseConst *__restrict__ cc, CaseDyn *__restrict__ dyn,
                         int nbits, State st, uint32_t *__restrict__ keys, int dst0,
                         const float *__restrict__ ghost) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const CaseConst &C = cc[slot];
  if (st.ghost)
    st.ghost[dst0 + i] = ghost ? make_float4(ghost[3 * i], ghost[3 * i + 1], ghost[3 * i + 2], 0.f)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
  int c[3];
  float off[3];
  bool inside = true;
  for (int k = 0; k < 3; k++) {
    // same cell rule as the oracle: floor((r - origin) / cs) in FP64
    double rel = pos[3 * i + k] - C.origin[k];
    double f = floor(rel / C.cs);
    int nk = k == 0 ? C.nx : (k == 1 ? C.ny : C.nz);
    if (!(f >= C.margin && f < nk - C.margin)) inside = false;
    c[k] = inside ? (int)f : 0;
    float o = (float)(rel - f * C.cs);
    if (o >= C.csf) o = below(C.csf);
    if (o < 0.f) o = 0.f;
    off[k] = o;
  }
  int d = dst0 + i;
  uint8_t code = type[i] == 0 ? 0 : (group && group[i] >= 0 ? (uint8_t)(2 + group[i]) : 1);
  float4 vr = make_float4(vel ? vel[3 * i] : 0.f, vel ? vel[3 * i + 1] : 0.f,
                          vel ? vel[3 * i + 2] : 0.f, rho[i]);
  uint32_t key;
  if (inside) {
    uint32_t lin = ((uint32_t)c[2] * C.ny + c[1]) * C.nx + c[0];
    key = key_make(C.cellbase + lin, code != 0, nbits);
    st.posc[d] = make_float4(off[0], off[1], off[2], (float)c[0]);
  } else {
    key = key_out(nbits);
    // frozen particles keep a float position relative to the grid origin
    st.posc[d] = make_float4((float)(pos[3 * i] - C.origin[0]),
                             (float)(pos[3 * i + 1] - C.origin[1]),
                             (float)(pos[3 * i + 2] - C.origin[2]), 0.f);
    atomicAdd(&dyn[slot].n_out, 1);
  }
  st.velrho[d] = vr;
  if (st.vrprev) st.vrprev[d] = vr;
  st.id[d] = id_base + (uint32_t)i;
  st.cid[d] = (uint16_t)slot;
  st.code[d] = code;
  keys[d] = key;
}

// ---- reorder + equation of state ------------------------------------------

// dst[i] = src[perm[i]]; the cell x index goes to posc.w and P/rho, with P
// the Tait pressure of Eq 28, to press[i].
__global__ void k_reorder(int n, const uint32_t *__restrict__ perm,
                          const uint32_t *__restrict__ keys_sorted,
                          const float4 *__restrict__ posc_src,
                          const float4 *__restrict__ velrho_src,
                          const uint32_t *__restrict__ id_src,
                          const uint16_t *__restrict__ cid_src,
                          const uint8_t *__restrict__ code_src,
                          const float4 *__restrict__ vrprev_src,
                          const float4 *__restrict__ ghost_src, State dst,
                          float *__restrict__ press, const CaseConst *__restrict__ cc,
                          CaseDyn *__restrict__ dyn, int nbits,
                          const float4 *__restrict__ ref_src = nullptr,
                          float4 *__restrict__ ref_dst = nullptr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int cidx = -1;
  unsigned v2 = 0u;
  if (i < n) {
    uint32_t p = perm[i];
    float4 pc = posc_src[p];
    float4 vr = velrho_src[p];
    cidx = cid_src[p];
    const CaseConst &C = cc[cidx];
    const uint32_t k = keys_sorted[i];
    if (k < key_out(nbits)) {
      const uint32_t lin = key_cell(k, nbits) - C.cellbase;
      pc.w = (float)(lin % (uint32_t)C.nx);
      v2 = __float_as_uint(fmaf(vr.x, vr.x, fmaf(vr.y, vr.y, vr.z * vr.z)));
    }
    dst.posc[i] = pc;
    dst.velrho[i] = vr;
    dst.id[i] = id_src[p];
    dst.cid[i] = (uint16_t)cidx;
    dst.code[i] = code_src[p];
    if (vrprev_src) dst.vrprev[i] = vrprev_src[p];
    if (ghost_src) dst.ghost[i] = ghost_src[p];
    if (ref_dst) ref_dst[i] = ref_src[p];  // kept list: build positions follow the order
    press[i] = tait_pressure(C, vr.w) / vr.w;
  }
  // max |v|^2 per case (for the neighbour list's skin): one atomic per warp
  // when the warp holds one case
  const unsigned full = 0xffffffffu;
  const int c0 = __shfl_sync(full, cidx, 0);
  if (__all_sync(full, cidx == c0)) {
    const unsigned m = __reduce_max_sync(full, v2);
    // (the maximum only grows: a warp whose value is not above the one it
    // reads, maybe an older one, leaves it; fewer same-address atomics)
    if ((threadIdx.x & 31) == 0 && c0 >= 0 && m &&
        m > *(volatile const unsigned *)&dyn[c0].v2max_bits)
      atomicMax(&dyn[c0].v2max_bits, m);
  } else if (cidx >= 0 && v2) {
    atomicMax(&dyn[cidx].v2max_bits, v2);
  }
}

// ---- restricted rebuild of the list kept across steps -----------------------
//
// At a rebuild event only the particles of the cases that need a new list are
// sorted again, when no index range can move (ctl->full == 0: no particle left
// the domain and no case was admitted or released since the last build).  A
// case's fluid particles then keep one fixed index range and its boundary
// particles another (all fluid keys lie below all boundary keys, and the cases
// follow their cellbase order), so the flagged particles, listed in index order
// and sorted stably by key, fill exactly the slots they came from: output p of
// that sort goes to the p-th flagged index.  With ctl->full every particle is
// flagged and the p-th flagged index is p: the full sort.  The other cases keep
// their order, cells and state untouched.
constexpr int kRbTile = 1024;

__device__ __forceinline__ bool rb_flag(int i, int n, const uint16_t *__restrict__ cid,
                                        const CaseDyn *__restrict__ dyn,
                                        const ListCtl *__restrict__ ctl) {
  return i < n && (ctl->full || dyn[cid[i]].need);
}

// The number of flagged particles in every tile of kRbTile indices.
__global__ void __launch_bounds__(kRbTile)
k_rb_count(int n, const uint16_t *__restrict__ cid, const CaseDyn *__restrict__ dyn,
           const ListCtl *__restrict__ ctl, uint32_t *__restrict__ tile_cnt) {
  const int i = blockIdx.x * kRbTile + threadIdx.x;
  const int c = __syncthreads_count(rb_flag(i, n, cid, dyn, ctl));
  if (threadIdx.x == 0) tile_cnt[blockIdx.x] = (uint32_t)c;
}

// One block: exclusive scan of the tile counts in place; the total to *m.
__global__ void __launch_bounds__(1024)
k_rb_scan(int ntiles, uint32_t *__restrict__ tile_cnt, int *__restrict__ m) {
  const unsigned full = 0xffffffffu;
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int base = 0; base < ntiles; base += 1024) {
    const int t = base + threadIdx.x;
    const uint32_t v = t < ntiles ? tile_cnt[t] : 0u;
    uint32_t x = v;  // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(full, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {  // inclusive scan of the warp totals
      uint32_t w = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(full, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = carry + (warp ? wsum[warp - 1] : 0u) + x - v;
    if (t < ntiles) tile_cnt[t] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *m = (int)carry;
}

// The flagged indices in index order (idx) and their keys (kc).
__global__ void __launch_bounds__(kRbTile)
k_rb_compact(int n, const uint16_t *__restrict__ cid, const CaseDyn *__restrict__ dyn,
             const ListCtl *__restrict__ ctl, const uint32_t *__restrict__ tile_off,
             const uint32_t *__restrict__ keys, uint32_t *__restrict__ idx,
             uint32_t *__restrict__ kc) {
  __shared__ uint32_t wcnt[kRbTile / 32];
  const int i = blockIdx.x * kRbTile + threadIdx.x;
  const bool f = rb_flag(i, n, cid, dyn, ctl);
  const unsigned b = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wcnt[warp] = (uint32_t)__popc(b);
  __syncthreads();
  if (!f) return;
  uint32_t off = tile_off[blockIdx.x];
  for (int w = 0; w < warp; w++) off += wcnt[w];
  const uint32_t p = off + (uint32_t)__popc(b & ((1u << lane) - 1u));
  idx[p] = (uint32_t)i;
  kc[p] = keys[i];
}

// k_reorder through the compaction: output p of the sort of the flagged keys
// (keys_sorted, perm) goes to slot idx[p] from the particle idx[perm[p]];
// keys_dst receives its key; the build positions follow (ref, kept list).
__global__ void k_rb_scatter(int n, const int *__restrict__ m_p, const uint32_t *__restrict__ idx,
                             const uint32_t *__restrict__ perm,
                             const uint32_t *__restrict__ keys_sorted, State src, State dst,
                             uint32_t *__restrict__ keys_dst, float *__restrict__ press,
                             const CaseConst *__restrict__ cc, CaseDyn *__restrict__ dyn,
                             int nbits, const float4 *__restrict__ ref_src,
                             float4 *__restrict__ ref_dst) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  int cidx = -1;
  unsigned v2 = 0u;
  if (p < n && p < *m_p) {
    const uint32_t d = idx[p], q = idx[perm[p]];
    float4 pc = src.posc[q];
    const float4 vr = src.velrho[q];
    cidx = src.cid[q];
    const CaseConst &C = cc[cidx];
    const uint32_t k = keys_sorted[p];
    if (k < key_out(nbits)) {
      const uint32_t lin = key_cell(k, nbits) - C.cellbase;
      pc.w = (float)(lin % (uint32_t)C.nx);
      v2 = __float_as_uint(fmaf(vr.x, vr.x, fmaf(vr.y, vr.y, vr.z * vr.z)));
    }
    keys_dst[d] = k;
    dst.posc[d] = pc;
    dst.velrho[d] = vr;
    dst.id[d] = src.id[q];
    dst.cid[d] = (uint16_t)cidx;
    dst.code[d] = src.code[q];
    if (src.vrprev) dst.vrprev[d] = src.vrprev[q];
    if (src.ghost) dst.ghost[d] = src.ghost[q];
    if (ref_dst) ref_dst[d] = ref_src[q];
    press[d] = tait_pressure(C, vr.w) / vr.w;
  }
  // max |v|^2 per case (for the skin of the cases that rebuild), as k_reorder
  const unsigned full = 0xffffffffu;
  const int c0 = __shfl_sync(full, cidx, 0);
  if (__all_sync(full, cidx == c0)) {
    const unsigned mx = __reduce_max_sync(full, v2);
    if ((threadIdx.x & 31) == 0 && c0 >= 0 && mx &&
        mx > *(volatile const unsigned *)&dyn[c0].v2max_bits)
      atomicMax(&dyn[c0].v2max_bits, mx);
  } else if (cidx >= 0 && v2) {
    atomicMax(&dyn[cidx].v2max_bits, v2);
  }
}

// ---- cell start table --------------------------------------------------------

// cstart (pre-filled with 0xff): first sorted index of every non-empty
// (type, cell); cstart[cap1-1] = end of the fluid segment, cstart[2 cap1-1] =
// nvalid (first out-of-domain / released key).
__global__ void k_mark(int n, const uint32_t *__restrict__ keys, uint32_t *__restrict__ cstart,
                       uint32_t cap1, int nbits, int *__restrict__ nvalid) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys[i], kout = key_out(nbits), bb = key_bbit(nbits);
  const uint32_t prev = i > 0 ? keys[i - 1] : 0u;
  if (k >= bb && (i == 0 || prev < bb)) cstart[cap1 - 1] = (uint32_t)i;
  if (i == n - 1 && k < bb) cstart[cap1 - 1] = (uint32_t)n;
  if (k >= kout && (i == 0 || prev < kout)) {
    *nvalid = i;
    cstart[2 * cap1 - 1] = (uint32_t)i;
  }
  if (i == n - 1 && k < kout) {
    *nvalid = n;
    cstart[2 * cap1 - 1] = (uint32_t)n;
  }
  if (k < kout && (i == 0 || prev != k))
    cstart[(key_boundary(k, nbits) ? cap1 : 0u) + key_cell(k, nbits)] = (uint32_t)i;
}

// Suffix minimum over cstart (empty cells take the start of the next
// non-empty one): per-block pass, carry pass, apply pass.
constexpr int kFillThreads = 1024, kFillItems = 4, kFillBlock = kFillThreads * kFillItems;

__device__ __forceinline__ uint32_t warp_suffix_min(uint32_t v) {
  const int lane = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v = min(v, y);
  }
  return v;
}

// In place: each block turns its chunk into a chunk-local suffix minimum and
// writes the chunk minimum to bmin.
__global__ void __launch_bounds__(kFillThreads)
k_fill_block(uint32_t *__restrict__ a, int64_t len, uint32_t *__restrict__ bmin) {
  __shared__ uint32_t wmin[32];
  const int64_t base = (int64_t)blockIdx.x * kFillBlock + (int64_t)threadIdx.x * kFillItems;
  uint32_t v[kFillItems];
  for (int q = 0; q < kFillItems; q++) v[q] = base + q < len ? a[base + q] : 0xffffffffu;
  for (int q = kFillItems - 2; q >= 0; q--) v[q] = min(v[q], v[q + 1]);
  const uint32_t s = warp_suffix_min(v[0]);  // inclusive suffix over the lanes of this warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wmin[warp] = s;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = wmin[lane];
    w = warp_suffix_min(w);
    wmin[lane] = w;  // inclusive suffix over warps
  }
  __syncthreads();
  uint32_t after = 0xffffffffu;  // minimum of everything after this thread's items
  const uint32_t nxt = __shfl_down_sync(0xffffffffu, s, 1);
  if (lane < 31) after = nxt;
  if (warp < 31) after = min(after, wmin[warp + 1]);
  for (int q = 0; q < kFillItems; q++)
    if (base + q < len) a[base + q] = min(v[q], after);
  if (threadIdx.x == 0) bmin[blockIdx.x] = wmin[0];
}

// Single block: bmin[b] <- min over the blocks after b (exclusive suffix min).
__global__ void __launch_bounds__(1024) k_fill_carry(uint32_t *__restrict__ bmin, int nb) {
  __shared__ uint32_t wmin[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0xffffffffu;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int end = nb; end > 0; end -= 1024) {  // chunks of 1024 from the end
    const int idx = end - 1024 + (int)threadIdx.x;
    const uint32_t v = idx >= 0 ? bmin[idx] : 0xffffffffu;
    const uint32_t s = warp_suffix_min(v);
    if (lane == 0) wmin[warp] = s;
    __syncthreads();
    if (warp == 0) wmin[lane] = warp_suffix_min(wmin[lane]);
    __syncthreads();
    uint32_t after = carry;
    const uint32_t nxt = __shfl_down_sync(0xffffffffu, s, 1);
    if (lane < 31) after = min(after, nxt);
    if (warp < 31) after = min(after, wmin[warp + 1]);
    const uint32_t chunk_min = wmin[0];
    __syncthreads();
    if (idx >= 0) bmin[idx] = after;
    if (threadIdx.x == 0) carry = min(carry, chunk_min);
    __syncthreads();
  }
}

__global__ void k_fill_apply(uint32_t *__restrict__ a, int64_t len,
                             const uint32_t *__restrict__ carry) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  const uint32_t c = carry[i / kFillBlock];
  if (c < a[i]) a[i] = c;
}

// ---- particle interaction ----------------------------------------------------

// npairs: all pairs of a; nfb: pairs with a in F, b in B; nbf: pairs with a in B.
__device__ __forceinline__ void reduce_case(int cidx, bool has, unsigned npairs, unsigned nfb,
                                            unsigned nbf, unsigned dtbits, bool bad,
                                            CaseDyn *dyn) {
  const unsigned full = 0xffffffffu;
  int c0 = __shfl_sync(full, cidx, 0);
  bool uniform = __all_sync(full, cidx == c0 && has);
  if (uniform) {
    unsigned p32 = __reduce_add_sync(full, npairs);
    unsigned fb = __reduce_add_sync(full, nfb);
    unsigned bf = __reduce_add_sync(full, nbf);
    unsigned m = __reduce_min_sync(full, dtbits);
    unsigned anybad = __any_sync(full, bad);
    if ((threadIdx.x & 31) == 0) {
      if (p32) atomicAdd(&dyn[c0].pairs, (unsigned long long)p32);
      if (fb) atomicAdd(&dyn[c0].pairs_fb, (unsigned long long)fb);
      if (bf) atomicAdd(&dyn[c0].pairs_bf, (unsigned long long)bf);
      if (m < kFloatInfBits) atomicMin(&dyn[c0].dtmin_bits, m);
      if (anybad) atomicOr(&dyn[c0].flags, kFlagNaN);
    }
  } else if (has) {
    if (npairs) atomicAdd(&dyn[cidx].pairs, (unsigned long long)npairs);
    if (nfb) atomicAdd(&dyn[cidx].pairs_fb, (unsigned long long)nfb);
    if (nbf) atomicAdd(&dyn[cidx].pairs_bf, (unsigned long long)nbf);
    if (dtbits < kFloatInfBits) atomicMin(&dyn[cidx].dtmin_bits, dtbits);
    if (bad) atomicOr(&dyn[cidx].flags, kFlagNaN);
  }
}

// Gap between an offset o in [0, cs) and the slab of cells at relative index d.
__device__ __forceinline__ float slab_gap(int d, float o, float cs) {
  return d > 0 ? fmaf((float)d, cs, -o) : (d < 0 ? o - (float)(d + 1) * cs : 0.f);
}

// Per-particle accumulators of one interaction evaluation.
struct Acc {
  float ax, ay, az;  // sum t^3 [(Pa+Pb)/rho_b + kv min(v.r,0)/((r^2+eta^2)(rho_a+rho_b))] r_ab
  float s1;          // sum t^3 / rho_b v_ab.r_ab            (continuity, Eq 15 / 36)
  float s2;          // sum_{b in F} t^3 / rho_b (rho_b - rho_a)  (density diffusion, Eq 17-18)
  float mur;         // max |v_ab.r_ab| / (r^2 + eta^2)      (Eq 35)
  unsigned cnt, cntb;
};

// Hydrostatic density difference rho^H_ab of Eq 19: Eq 28 solved for the
// density at the pressure P^H_ab = rho0 g z_ab of Eq 20, minus rho0, i.e.
// rho0 ((1 + x)^k - 1) with x = P^H_ab / B and k = 1/gamma.  Within the
// kernel support |x| is small (|x| <= 2h gamma |g| / cs0^2, about 1e-3 for
// the usual cs0), where the binomial series to x^4 is used: its first
// omitted term is below 2e-9 relative for |x| < 1e-2; otherwise log1p/expm1.
__device__ __forceinline__ float rho_hydro(const CaseConst &C, float rx, float ry, float rz) {
  const float x = fmaf(C.khyd[0], rx, fmaf(C.khyd[1], ry, C.khyd[2] * rz));  // P^H / B
  if (fabsf(x) < 1e-2f) {
    const float s = fmaf(C.hyd_c[0] * x, fmaf(C.hyd_c[1] * x, fmaf(C.hyd_c[2], x, 1.f), 1.f), 1.f);
    return C.rho0 * C.inv_gamma * x * s;
  }
  return C.rho0 * expm1f(log1pf(x) * C.inv_gamma);
}

// Per-target data of the physics beyond the default model: Eq 19-20 density
// diffusion (hyd) and laminar viscosity + SPS stress (sps, Eq 23-27).
struct Ext {
  const CaseConst *C;
  bool hyd, sps;
  float kl;      // -4 nu0 rho_a (Eq 23, in the units of the momentum sums)
  float ta[6];   // rho_a (tau/rho)_a: xx, yy, zz, xy, xz, yz (Eq 25)
  const float4 *__restrict__ tau4;  // (tau/rho)_b: xx, yy, zz, xy
  const float2 *__restrict__ tau2;  // (tau/rho)_b: xz, yz
};

// Pair terms for a fluid particle a and a neighbour b (ddt: b in F).
// grad_a W_ab = cw t^3 r_ab with t = 1 - r/(2h) (derivative of Eq 11).
// Qb = P_b / rho_b, so (P_a + P_b) / rho_b = P_a / rho_b + Qb.  All momentum
// terms are summed in units of -rho_a / (m cw), like the pressure term.
// EXT = 0 compiles the Eq 19 and Eq 23-27 branches out, 1 keeps Eq 19, 2
// both; X describes target a and j is b's index (bfluid: b in F).
template <int EXT = 0>
__device__ __forceinline__ void pair_fluid(const float4 &va, float Pa, float kv, float hih,
                                           float eta2, float rx, float ry, float rz, float r2,
                                           const float4 &vb, float Qb, bool ddt, Acc &A,
                                           const Ext *X = nullptr, int j = 0,
                                           bool bfluid = true) {
  const float rr = r2 * rsqrtf(r2);
  const float t = fmaf(-hih, rr, 1.f);
  const float t3 = t * t * t;
  const float vx = va.x - vb.x, vy = va.y - vb.y, vz = va.z - vb.z;
  const float vr = fmaf(vx, rx, fmaf(vy, ry, vz * rz));
  const float ib = __fdividef(1.f, vb.w);
  const float w = t3 * ib;
  A.s1 = fmaf(w, vr, A.s1);
  if (ddt) {
    float d = vb.w - va.w;
    if (EXT >= 1 && X->hyd) d -= rho_hydro(*X->C, rx, ry, rz);
    A.s2 = fmaf(w, d, A.s2);
  }
  const float sab = va.w + vb.w;
  const float ie = __fdividef(1.f, (r2 + eta2) * sab);
  const float mu = vr * ie * sab;  // v_ab.r_ab / (r^2 + eta^2)
  A.mur = fmaxf(A.mur, fabsf(mu));
  const float pi = fminf(vr, 0.f) * ie;
  const float u = fmaf(kv, pi, fmaf(Pa, ib, Qb));
  const float s = t3 * u;
  A.ax = fmaf(s, rx, A.ax);
  A.ay = fmaf(s, ry, A.ay);
  A.az = fmaf(s, rz, A.az);
  if (EXT == 2 && X->sps) {
    // Eq 23: m 4 nu0 (r.gradW) v_ab / ((rho_a + rho_b)(r^2 + eta^2)), r.gradW = cw t^3 r^2
    const float cl = X->kl * t3 * r2 * ie;
    A.ax = fmaf(cl, vx, A.ax);
    A.ay = fmaf(cl, vy, A.ay);
    A.az = fmaf(cl, vz, A.az);
    // Eq 26: m (tau_a + tau_b)^{ij} / (rho_a rho_b) grad^j W with tau = rho (tau/rho);
    // boundary particles carry no SPS stress
    const float4 b4 = bfluid ? X->tau4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 b2 = bfluid ? X->tau2[j] : make_float2(0.f, 0.f);
    const float txx = fmaf(X->ta[0], ib, b4.x), tyy = fmaf(X->ta[1], ib, b4.y);
    const float tzz = fmaf(X->ta[2], ib, b4.z), txy = fmaf(X->ta[3], ib, b4.w);
    const float txz = fmaf(X->ta[4], ib, b2.x), tyz = fmaf(X->ta[5], ib, b2.y);
    A.ax = fmaf(-t3, fmaf(txx, rx, fmaf(txy, ry, txz * rz)), A.ax);
    A.ay = fmaf(-t3, fmaf(txy, rx, fmaf(tyy, ry, tyz * rz)), A.ay);
    A.az = fmaf(-t3, fmaf(txz, rx, fmaf(tyz, ry, tzz * rz)), A.az);
  }
}

// Boundary particle a: continuity over fluid neighbours only (Eq 36).
__device__ __forceinline__ void pair_boundary(const float4 &va, float hih, float rx, float ry,
                                              float rz, float r2, const float4 &vb, Acc &A) {
  const float rr = r2 * rsqrtf(r2);
  const float t = fmaf(-hih, rr, 1.f);
  const float t3 = t * t * t;
  const float vx = va.x - vb.x, vy = va.y - vb.y, vz = va.z - vb.z;
  const float vr = fmaf(vx, rx, fmaf(vy, ry, vz * rz));
  A.s1 = fmaf(t3 * __fdividef(1.f, vb.w), vr, A.s1);
}

// Final values of target a from its accumulators: dv/dt (Eq 22 with g), drho/dt
// (Eq 15 with the Eq 17-18 term, or Eq 36), mu_max and the Eq 35 candidate
// time step; then the warp's per-case reduction of counts, dt and flags.
// With several lanes per target (all holding the same totals) only the lead
// lane writes and counts.
__device__ __forceinline__ void finish_target(const CaseConst &C, int i, int n, int cidx, bool has,
                                              bool afluid, const float4 &va, const Acc &A,
                                              int want_dt, float4 *__restrict__ ace,
                                              float *__restrict__ mu_out, CaseDyn *dyn,
                                              bool lead = true) {
  unsigned npairs = 0, nfb = 0, nbf = 0, dtbits = kFloatInfBits;
  bool bad = false;
  if (has) {
    npairs = A.cnt + A.cntb;
    nfb = afluid ? A.cntb : 0u;
    nbf = afluid ? 0u : A.cnt;
    const float mcw = C.m * C.cw;
    float4 out;
    float mumax = C.h * A.mur;
    if (afluid) {
      const float ca = -mcw / va.w;
      out.x = fmaf(ca, A.ax, C.g[0]);
      out.y = fmaf(ca, A.ay, C.g[1]);
      out.z = fmaf(ca, A.az, C.g[2]);
      out.w = mcw * (va.w * A.s1 - C.kddt * A.s2);
      const float f = sqrtf(out.x * out.x + out.y * out.y + out.z * out.z);
      const float dtf = f > 0.f ? sqrtf(C.h / f) : INFINITY;
      const float dtcv = C.h / (C.cs0f + mumax);
      bad = !(isfinite(out.x) && isfinite(out.y) && isfinite(out.z) && isfinite(out.w));
      if (want_dt) dtbits = __float_as_uint(fminf(dtf, dtcv));
    } else {
      out = make_float4(0.f, 0.f, 0.f, mcw * va.w * A.s1);
      mumax = 0.f;
      bad = !isfinite(out.w);
    }
    if (lead) {
      ace[i] = out;
      if (mu_out) mu_out[i] = mumax;
    } else {
      npairs = nfb = nbf = 0u;
    }
  }
  reduce_case(i < n ? cidx : -1, has, npairs, nfb, nbf, dtbits, bad, dyn);
}

// Skin of a list built on state n, per case (k_list_begin): the largest
// approach of two particles over one step, dt |v|max x 1.25 with dt bounded
// by Eq 35 (dt <= C_CFL h / cs0 since dt_cv <= h / cs0) or the fixed step,
// plus 1e-3 h; the 25 % covers the change of a wall's imposed speed over
// dt / 2.  A list kept across steps adds extra x 2h.  The build's rows reach
// 2h + cs, so the skin is capped at 0.95 cs (kFlagSkin if one step needs more).
// Also sets each case's build mode: with fresh_all (one list per step) every
// case builds from its state; else a case that needs a rebuild does (and
// takes a new skin), one whose particles moved in the sorted order (another
// case's particle left the domain, a case was admitted or released) rebuilds
// its records from its build positions with its old skin, and the rest keep
// their records.  Clears the rebuild request and counts the build.
__global__ void k_list_begin(int ncases, const CaseConst *__restrict__ cc,
                             CaseDyn *__restrict__ dyn, ListCtl *__restrict__ ctl, float extra,
                             int fresh_all, const uint32_t *__restrict__ cstart, uint32_t cap1) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c == 0 && ctl) {
    ctl->rebuild = 0u;
    ctl->full = 0u;
    ctl->builds += 1ull;
  }
  if (c >= ncases || !cc[c].active) return;
  const CaseConst &C = cc[c];
  CaseDyn &D = dyn[c];
  const uint32_t sF = cstart[C.cellbase], sB = cstart[cap1 + C.cellbase];
  if (fresh_all || D.need) {
    const float need = fmaf(C.list_k, sqrtf(__uint_as_float(D.v2max_bits)), 1e-3f * C.h);
    const float smax = 0.95f * C.csf;
    if (need > smax) D.flags |= kFlagSkin;
    D.skin = fminf(fmaf(extra, 2.f * C.h, need), smax);
    D.lmode = 1u;
  } else {
    D.lmode = (sF != D.startF || sB != D.startB) ? 2u : 0u;
  }
  D.need = 0u;
  D.startF = sF;
  D.startB = sB;
}

// Before the sort of a kept-list rebuild that re-sorts every case (ctl->full):
// the cases that need no rebuild enter it with their build keys and their
// state in the build's cells (y), so that they keep their particle order and
// cells; the others with the normalised state the corrector wrote into x.
// (A restricted rebuild sorts only the cases that need one: nothing to do.)
__global__ void k_select(int n, const uint16_t *__restrict__ cid,
                         const CaseConst *__restrict__ cc, const CaseDyn *__restrict__ dyn,
                         const uint32_t *__restrict__ keys_build, const float4 *__restrict__ posc_build,
                         uint32_t *__restrict__ keys, float4 *__restrict__ posc,
                         const ListCtl *__restrict__ ctl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !ctl->full) return;
  const int c = cid[i];
  if (!cc[c].active || dyn[c].need) return;
  keys[i] = keys_build[i];
  posc[i] = posc_build[i];
}

// Marks every case's list for a rebuild (after the sorted state was
// overwritten outside the step, or the pair loop changed).
__global__ void k_need_all(int ncases, CaseDyn *__restrict__ dyn) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncases) dyn[c].need = 1u;
}

// One thread per particle a in sorted order (all fluid targets first, then
// boundary targets, so warps rarely mix the two).  The (2M+1)^2 rows of
// neighbour cells (fixed dy, dz) are visited in lock-step by the warp; in a
// row each lane keeps only the cells that its own sphere of radius 2h can
// reach, which form one contiguous index range per particle type.
//
// VARIANT 0 (compacted): the candidates of a row are tested in chunks of 32
//   (r^2 < (2h)^2 only); the hits form a 32-bit mask per lane and the pair
//   terms then run over the set bits, so no lane idles on a rejected
//   candidate while another computes a pair.
// VARIANT 1 (inline): test and pair terms in one loop (divergent).
// (VARIANT 2, the queued pair loop, is k_interact_q below.)
// EXT (VARIANT 0 only): 1 adds the Eq 19-20 density diffusion, 2 also the
// laminar + SPS viscosity of Eq 23-27 (tau4/tau2 from k_strain), per case;
// warps without such cases still take the default pair loop.
//
// LIST (VARIANT 0): 1 also writes the target's neighbour list, 2 writes
// only the list (no pair terms, no outputs besides the list and ref): for
// every tested chunk with a candidate within 2h + skin, one record (first
// index | row offset, mask of those candidates) to list[i cap + c] (a target's
// records side by side, four to a 32-byte sector), at most cap per target.  The
// list's rows reach one cell further than the 2h support (M + 1 cells, so
// 2h + cs >= 2h + skin), clipped to the case's grid.  ref, if set, receives
// the target's position at the build (the list kept across steps), and the
// case's build mode applies (k_list_begin): 0 keeps the target's records, 1
// builds from posc, 2 rebuilds from the previous build positions (ref_src,
// gathered into the new order) with the case's old skin.  3 is 2 with only
// the candidates of larger index than the target (the half list of the
// pair-once walk: a boundary target, after every fluid index, gets none).
// LIST | 4 (6, 7): wide records, the whole 32-bit first index with no row
// code (engines beyond 2^25 particles; the walks find the row from the
// first candidate's cell).
template <int M, int VARIANT, int EXT = 0, int LIST = 0>
__global__ void __launch_bounds__(128, EXT == 2 ? 6 : 0)
k_interact(int n, const int *__restrict__ nvalid_p, const uint32_t *__restrict__ keys,
           const float4 *__restrict__ posc, const float4 *__restrict__ velrho,
           const float *__restrict__ press, const uint16_t *__restrict__ cid,
           const uint32_t *__restrict__ cstart, uint32_t cap1, int nbits,
           const CaseConst *__restrict__ cc, CaseDyn *__restrict__ dyn,
           float4 *__restrict__ ace, float *__restrict__ mu_out, int want_dt,
           const float4 *__restrict__ tau4 = nullptr, const float2 *__restrict__ tau2 = nullptr,
           uint2 *__restrict__ list = nullptr, int cap = 0,
           uint16_t *__restrict__ count = nullptr, float4 *__restrict__ ref = nullptr,
           const float4 *__restrict__ ref_src = nullptr) {
  const unsigned full = 0xffffffffu;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nvalid = *nvalid_p;
  const bool has = i < nvalid;
  const int cidx = i < n ? (int)cid[i] : 0;
  const CaseConst &C = cc[cidx];
  const uint32_t key = has ? keys[i] : 0u;
  const bool afluid = has && !key_boundary(key, nbits);
  const int gc = (int)key_cell(key, nbits);
  const int nx = C.nx, nxy = C.nx * C.ny;
  const float cs = C.csf, ics = C.inv_csf, r2max = C.r2max, eta2 = C.eta2, hih = C.half_inv_h;
  // 0 < r2 < r2max as one unsigned compare (r2 >= 0; +0 wraps to UINT_MAX)
  const unsigned r2max_u = __float_as_uint(r2max) - 1u;
  float r2l = r2max;  // list radius^2: (2h + skin)^2 with LIST
  int tcx = 0, tcy = 0, tcz = 0;  // LIST: the target's cell, for the grid clip
  if (LIST) {
    const float R = sqrtf(r2max) + dyn[cidx].skin;
    r2l = R * R;
    if (has) decode_cell((uint32_t)gc - C.cellbase, nx, C.ny, tcx, tcy, tcz);
  }
  const unsigned r2l_u = __float_as_uint(r2l) - 1u;
  const float r2prune = r2l * 1.0001f;  // conservative: pruning never drops a pair
  int lcnt = 0;                          // LIST: records written
  const int lmode = (LIST >= 2 && ref) ? (int)dyn[cidx].lmode : 1;
  const float4 *__restrict__ P = lmode == 2 ? ref_src : posc;  // positions walked
  const float4 pa = has ? P[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 va = has ? velrho[i] : make_float4(0.f, 0.f, 0.f, 1.f);
  const float Pa = has ? press[i] * va.w : 0.f;  // press holds P / rho
  const float kv = C.kvisc * va.w;
  const bool ddt_on = C.ddt != 0;
  // boundary targets of an mDBC case take their density from Eq 38, not Eq 36;
  // a half list (every boundary index above every fluid one) leaves boundary
  // targets without candidates
  constexpr bool HALF = (LIST & 3) == 3;
  const bool work = has && (afluid || C.bmode == 0) && lmode != 0 && (!HALF || afluid);
  Ext X;
  X.C = &C;
  X.hyd = EXT >= 1 && C.ddt == 2;
  X.sps = EXT == 2 && C.visc == 1 && afluid;
  X.kl = -4.f * C.nu0 * va.w;
  X.tau4 = tau4;
  X.tau2 = tau2;
  {
    const float4 t4 = X.sps ? tau4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 t2 = X.sps ? tau2[i] : make_float2(0.f, 0.f);
    X.ta[0] = va.w * t4.x;
    X.ta[1] = va.w * t4.y;
    X.ta[2] = va.w * t4.z;
    X.ta[3] = va.w * t4.w;
    X.ta[4] = va.w * t2.x;
    X.ta[5] = va.w * t2.y;
  }
  const bool warp_plain = __all_sync(full, (afluid || !has) && !X.hyd && !X.sps);
  Acc A = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u};
  constexpr int MR = LIST ? M + 1 : M;  // rows reach MR cells
  // the build position: taken now (mode 1), gathered into the new order by
  // the sort (mode 2), or kept where it is (mode 0: the target did not move)
  if (LIST && ref && i < n && lmode != 0) ref[i] = lmode == 1 ? pa : ref_src[i];
  // rows dy, dz in [-M, M]; a list build adds row -(M+1) (M+1) for the
  // targets within the skin of their cell's lower (upper) face, over the
  // warp's union of those ranges
  int ylo = -M, yhi = M, zlo = -M, zhi = M;
  if (LIST) {
    // row -(M+1) lies within the list radius iff o < R - M cs (R rounded up)
    const float sk = fmaf(-(float)M, cs, sqrtf(r2prune) * 1.0001f);
    const bool w = work;
    ylo = __reduce_min_sync(full, (w && pa.y < sk) ? -MR : -M);
    yhi = __reduce_max_sync(full, (w && pa.y > cs - sk) ? MR : M);
    zlo = __reduce_min_sync(full, (w && pa.z < sk) ? -MR : -M);
    zhi = __reduce_max_sync(full, (w && pa.z > cs - sk) ? MR : M);
  }
  const int wy = yhi - ylo + 1, nrows = wy * (zhi - zlo + 1);

#pragma unroll 1
  for (int row = 0; row < nrows; row++) {
    const int dy = ylo + row % wy, dz = zlo + row / wy;
    const float gy = slab_gap(dy, pa.y, cs), gz = slab_gap(dz, pa.z, cs);
    const float d2 = fmaf(gy, gy, gz * gz);
    int loF = 0, hiF = 0, loB = 0, hiB = 0;
    // the outer rows of a list build stay inside the case's grid
    const bool inrow = !LIST || (tcy + dy >= 0 && tcy + dy < C.ny && tcz + dz >= 0 &&
                                 tcz + dz < C.nz);
    if (work && inrow && d2 < r2prune) {
      const float L = sqrtf(r2prune - d2);
      int kx0 = max(-MR, (int)floorf((pa.x - L) * ics));
      int kx1 = min(MR, (int)floorf((pa.x + L) * ics));
      if (LIST) {
        kx0 = max(kx0, -tcx);
        kx1 = min(kx1, nx - 1 - tcx);
      }
      const int c0 = gc + dz * nxy + dy * nx + kx0;
      const int c1 = gc + dz * nxy + dy * nx + kx1 + 1;
      // half list: the fluid particles of the rows below the target's and of
      // the cells before its own in its row have smaller indices (cell order)
      const bool below = HALF && (dz < 0 || (dz == 0 && dy < 0));
      if (!below) {
        loF = (int)cstart[HALF && dz == 0 && dy == 0 ? gc + max(kx0, 0) : c0];
        hiF = (int)cstart[c1];
      }
      if (afluid) {
        loB = (int)cstart[cap1 + c0];
        hiB = (int)cstart[cap1 + c1];
      }
    }
    const float sy = fmaf(-(float)dy, cs, pa.y), sz = fmaf(-(float)dz, cs, pa.z);
    const uint32_t rowbits = list_row_code(dy, dz);
#pragma unroll 1
    for (int part = 0; part < 2; part++) {  // fluid neighbours, then boundary neighbours
      const int lo = part ? loB : loF;
      const int len = (part ? hiB : hiF) - lo;
      const int maxlen = (int)__reduce_max_sync(full, (unsigned)max(len, 0));
      const bool ddt = ddt_on && part == 0;
#pragma unroll 1
      for (int base = 0; base < maxlen; base += 32) {
        if (VARIANT == 0) {
          unsigned m = 0u, ml = 0u;
          const int nk = min(32, maxlen - base);
#pragma unroll 8
          for (int k = 0; k < nk; k++) {
            if (base + k < len) {
              const float4 pb = P[lo + base + k];
              const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
              const float ry = sy - pb.y, rz = sz - pb.z;
              const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
              if (__float_as_uint(r2) - 1u < r2max_u) m |= 1u << k;
              if (LIST && __float_as_uint(r2) - 1u < r2l_u) ml |= 1u << k;
            }
          }
          if ((LIST & 3) == 3) {  // half list: only candidates of larger index than the target
            const int lowk = i - (lo + base) + 1;
            if (lowk > 0) ml = lowk >= 32 ? 0u : ml & (0xffffffffu << lowk);
          }
          if (LIST && ml) {
            if (lcnt < cap)
              list[(int64_t)i * cap + lcnt] =
                  make_uint2((uint32_t)(lo + base) | (LIST & 4 ? 0u : rowbits), ml);
            lcnt++;
          }
          if (LIST < 2) {
          if (part) A.cntb += __popc(m); else A.cnt += __popc(m);
          if (warp_plain) {  // fluid targets, Eq 18 or no diffusion
            while (__any_sync(full, m != 0u)) {
              if (m) {
                const int k = 31 - __clz(m);
                m ^= 1u << k;
                const int j = lo + base + k;
                const float4 pb = posc[j];
                const float4 vb = velrho[j];
                const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
                const float ry = sy - pb.y, rz = sz - pb.z;
                const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                pair_fluid<false>(va, Pa, kv, hih, eta2, rx, ry, rz, r2, vb, press[j], ddt, A);
              }
            }
          } else {
            while (__any_sync(full, m != 0u)) {
              if (m) {
                const int k = 31 - __clz(m);
                m ^= 1u << k;
                const int j = lo + base + k;
                const float4 pb = posc[j];
                const float4 vb = velrho[j];
                const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
                const float ry = sy - pb.y, rz = sz - pb.z;
                const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                if (afluid)
                  pair_fluid<EXT>(va, Pa, kv, hih, eta2, rx, ry, rz, r2, vb, press[j], ddt, A,
                                  &X, j, part == 0);
                else
                  pair_boundary(va, hih, rx, ry, rz, r2, vb, A);
              }
            }
          }
          }
        } else {
          const int nk = min(32, maxlen - base);
#pragma unroll 1
          for (int k = 0; k < nk; k++) {
            if (base + k < len) {
              const int j = lo + base + k;
              const float4 pb = posc[j];
              const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
              const float ry = sy - pb.y, rz = sz - pb.z;
              const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
              if (__float_as_uint(r2) - 1u < r2max_u) {
                const float4 vb = velrho[j];
                if (afluid) {
                  pair_fluid(va, Pa, kv, hih, eta2, rx, ry, rz, r2, vb, press[j], ddt, A);
                  if (part) A.cntb++; else A.cnt++;
                } else {
                  pair_boundary(va, hih, rx, ry, rz, r2, vb, A);
                  A.cnt++;
                }
              }
            }
          }
        }
      }
    }
  }

  if (LIST && i < n && lmode != 0) {
    count[i] = (uint16_t)min(lcnt, cap);
    if (has && lcnt > cap) atomicOr(&dyn[cidx].flags, kFlagListFull);
  }
  if (LIST >= 2) return;
  finish_target(C, i, n, cidx, has, afluid, va, A, want_dt, ace, mu_out, dyn);
}

// Queued pair loop (VARIANT 2).  Same rows, pruning and 32-candidate test as
// VARIANT 0, but a chunk's hits are not evaluated at once: each lane appends
// (first index, hit mask, row, part) to its own FIFO in shared memory, and the
// warp evaluates one pair per lane per iteration only while every active lane
// has a queued hit.  A lane's hits from many rows are thus evaluated back to
// back, so the warp's lock-step waste follows the imbalance of whole neighbour
// counts rather than that of every row.  Each lane still takes its pairs in the
// same order as VARIANT 0, so the sums are bit-identical to it.
constexpr int kQCap = 16;  // FIFO slots per lane (power of two)

template <int M>
__global__ void __launch_bounds__(128, 6)
k_interact_q(int n, const int *__restrict__ nvalid_p, const uint32_t *__restrict__ keys,
             const float4 *__restrict__ posc, const float4 *__restrict__ velrho,
             const float *__restrict__ press, const uint16_t *__restrict__ cid,
             const uint32_t *__restrict__ cstart, uint32_t cap1, int nbits,
             const CaseConst *__restrict__ cc, CaseDyn *__restrict__ dyn,
             float4 *__restrict__ ace, float *__restrict__ mu_out, int want_dt) {
  __shared__ uint32_t q_base[kQCap * 128];
  __shared__ uint32_t q_mask[kQCap * 128];
  __shared__ uint8_t q_row[kQCap * 128];  // row | part << 7
  const unsigned full = 0xffffffffu;
  const int tid = threadIdx.x;
  const int i = blockIdx.x * blockDim.x + tid;
  const int nvalid = *nvalid_p;
  const bool has = i < nvalid;
  const int cidx = i < n ? (int)cid[i] : 0;
  const CaseConst &C = cc[cidx];
  const uint32_t key = has ? keys[i] : 0u;
  const bool afluid = has && !key_boundary(key, nbits);
  const int gc = (int)key_cell(key, nbits);
  const int nx = C.nx, nxy = C.nx * C.ny;
  const float cs = C.csf, ics = C.inv_csf, r2max = C.r2max, eta2 = C.eta2, hih = C.half_inv_h;
  const float r2prune = r2max * 1.0001f;
  const unsigned r2max_u = __float_as_uint(r2max) - 1u;
  const float4 pa = has ? posc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 va = has ? velrho[i] : make_float4(0.f, 0.f, 0.f, 1.f);
  const float Pa = has ? press[i] * va.w : 0.f;
  const float kv = C.kvisc * va.w;
  const bool ddt_on = C.ddt != 0;
  const bool work = has && (afluid || C.bmode == 0);
  const bool warp_fluid = __all_sync(full, afluid || !has);
  const unsigned active = __ballot_sync(full, has);
  Acc A = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u};
  constexpr int W = 2 * M + 1;

  // FIFO state of this lane and the entry being evaluated
  unsigned head = 0, tail = 0;
  unsigned cur = 0u;
  int cbase = 0;
  float csy = 0.f, csz = 0.f;
  bool cddt = false;

  // one pair of this lane (if it has one): pop an entry when the current is done
  auto pair_step = [&]() {
    if (cur == 0u && head != tail) {
      const int s = (int)(head & (kQCap - 1)) * 128 + tid;
      cur = q_mask[s];
      cbase = (int)q_base[s];
      const int rw = q_row[s];
      head++;
      const int r = rw & 0x7f;
      csy = fmaf(-(float)(r % W - M), cs, pa.y);
      csz = fmaf(-(float)(r / W - M), cs, pa.z);
      cddt = ddt_on && !(rw & 0x80);
    }
    if (cur) {
      const int k = 31 - __clz(cur);
      cur ^= 1u << k;
      const int j = cbase + k;
      const float4 pb = posc[j];
      const float4 vb = velrho[j];
      const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
      const float ry = csy - pb.y, rz = csz - pb.z;
      const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      if (warp_fluid || afluid)
        pair_fluid(va, Pa, kv, hih, eta2, rx, ry, rz, r2, vb, press[j], cddt, A);
      else
        pair_boundary(va, hih, rx, ry, rz, r2, vb, A);
    }
  };

#pragma unroll 1
  for (int row = 0; row < W * W; row++) {
    const int dy = row % W - M, dz = row / W - M;
    const float gy = slab_gap(dy, pa.y, cs), gz = slab_gap(dz, pa.z, cs);
    const float d2 = fmaf(gy, gy, gz * gz);
    int loF = 0, hiF = 0, loB = 0, hiB = 0;
    if (work && d2 < r2prune) {
      const float L = sqrtf(r2prune - d2);
      const int kx0 = max(-M, (int)floorf((pa.x - L) * ics));
      const int kx1 = min(M, (int)floorf((pa.x + L) * ics));
      const int c0 = gc + dz * nxy + dy * nx + kx0;
      const int c1 = gc + dz * nxy + dy * nx + kx1 + 1;
      loF = (int)cstart[c0];
      hiF = (int)cstart[c1];
      if (afluid) {
        loB = (int)cstart[cap1 + c0];
        hiB = (int)cstart[cap1 + c1];
      }
    }
    const float sy = fmaf(-(float)dy, cs, pa.y), sz = fmaf(-(float)dz, cs, pa.z);
#pragma unroll 1
    for (int part = 0; part < 2; part++) {
      const int lo = part ? loB : loF;
      const int len = (part ? hiB : hiF) - lo;
      const int maxlen = (int)__reduce_max_sync(full, (unsigned)max(len, 0));
#pragma unroll 1
      for (int base = 0; base < maxlen; base += 32) {
        unsigned m = 0u;
        const int nk = min(32, maxlen - base);
#pragma unroll 8
        for (int k = 0; k < nk; k++) {
          if (base + k < len) {
            const float4 pb = posc[lo + base + k];
            const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
            const float ry = sy - pb.y, rz = sz - pb.z;
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            if (__float_as_uint(r2) - 1u < r2max_u) m |= 1u << k;
          }
        }
        if (part) A.cntb += __popc(m); else A.cnt += __popc(m);
        // make room for this entry: a lane with a full FIFO evaluates (rare)
        while (__any_sync(full, m != 0u && tail - head >= (unsigned)kQCap)) pair_step();
        if (m) {
          const int s = (int)(tail & (kQCap - 1)) * 128 + tid;
          q_base[s] = (uint32_t)(lo + base);
          q_mask[s] = m;
          q_row[s] = (uint8_t)(row | (part << 7));
          tail++;
        }
        // balanced evaluation: one pair per lane while every active lane has one
        for (;;) {
          const unsigned busy = __ballot_sync(full, cur != 0u || head != tail);
          if (busy == 0u || (active & ~busy) != 0u) break;
          pair_step();
        }
      }
    }
  }
  while (__any_sync(full, cur != 0u || head != tail)) pair_step();
  finish_target(C, i, n, cidx, has, afluid, va, A, want_dt, ace, mu_out, dyn);
}

// Warp-shared candidate tiles (pi_variant 6): the lanes of a warp whose
// targets lie in one row of cells (same cell y and z of the same case) walk
// the union of their candidate ranges together.  Per row of neighbour cells
// the candidates [lo, hi) of the union are staged 32 at a time in shared
// memory, one coalesced load per array (position, velocity-density, P/rho),
// and every lane tests each staged candidate (a broadcast read) against its
// own target and evaluates the pairs inside 2h.  A candidate lies in one
// absolute row, visited once per group, so every pair is taken once; the
// exact cut-off test makes the pair set that of the other walks.
template <int M>
__global__ void __launch_bounds__(128)
k_interact_tile(int n, const int *__restrict__ nvalid_p, const uint32_t *__restrict__ keys,
                const float4 *__restrict__ posc, const float4 *__restrict__ velrho,
                const float *__restrict__ press, const uint16_t *__restrict__ cid,
                const uint32_t *__restrict__ cstart, uint32_t cap1, int nbits,
                const CaseConst *__restrict__ cc, CaseDyn *__restrict__ dyn,
                float4 *__restrict__ ace, float *__restrict__ mu_out, int want_dt) {
  __shared__ float4 t_pos[128];
  __shared__ float4 t_vel[128];
  __shared__ float t_q[128];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int wb = threadIdx.x & ~31;  // the warp's slice of the tiles
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nvalid = *nvalid_p;
  const bool has = i < nvalid;
  const int cidx = i < n ? (int)cid[i] : 0;
  const CaseConst &C = cc[cidx];
  const uint32_t key = has ? keys[i] : 0u;
  const bool afluid = has && !key_boundary(key, nbits);
  const int gc = (int)key_cell(key, nbits);
  const int nx = C.nx, nxy = C.nx * C.ny;
  const float cs = C.csf, ics = C.inv_csf, r2max = C.r2max, eta2 = C.eta2, hih = C.half_inv_h;
  const float r2prune = r2max * 1.0001f;
  const unsigned r2max_u = __float_as_uint(r2max) - 1u;
  const float4 pa = has ? posc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 va = has ? velrho[i] : make_float4(0.f, 0.f, 0.f, 1.f);
  const float Pa = has ? press[i] * va.w : 0.f;
  const float kv = C.kvisc * va.w;
  const bool ddt_on = C.ddt != 0;
  const bool work = has && (afluid || C.bmode == 0);
  // the cell of x = 0 in the target's row of cells: the group key
  const int cx = has ? (gc - (int)C.cellbase) % nx : 0;
  const int rowkey = work ? gc - cx : -1;
  Acc A = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u};
  constexpr int W = 2 * M + 1;

  unsigned todo = __ballot_sync(full, work);
#pragma unroll 1
  while (todo) {
    const int key0 = __shfl_sync(full, rowkey, __ffs(todo) - 1);
    const unsigned gmask = __ballot_sync(full, work && rowkey == key0);
    todo &= ~gmask;
    const bool in = (gmask >> lane) & 1u;
    const bool gfluid = __any_sync(full, in && afluid);
#pragma unroll 1
    for (int row = 0; row < W * W; row++) {
      const int dy = row % W - M, dz = row / W - M;
      const float gy = slab_gap(dy, pa.y, cs), gz = slab_gap(dz, pa.z, cs);
      const float d2 = fmaf(gy, gy, gz * gz);
      const bool reach = in && d2 < r2prune;  // this lane's sphere reaches the row
      int c0 = INT_MAX, c1 = INT_MIN;
      if (reach) {
        const float L = sqrtf(r2prune - d2);
        const int kx0 = max(-M, (int)floorf((pa.x - L) * ics));
        const int kx1 = min(M, (int)floorf((pa.x + L) * ics));
        c0 = gc + dz * nxy + dy * nx + kx0;
        c1 = gc + dz * nxy + dy * nx + kx1 + 1;
      }
      // the group's union of cells in this row (one contiguous range)
      const int u0 = __reduce_min_sync(full, c0);
      const int u1 = __reduce_max_sync(full, c1);
      if (u0 >= u1) continue;
      const float sy = fmaf(-(float)dy, cs, pa.y), sz = fmaf(-(float)dz, cs, pa.z);
#pragma unroll 1
      for (int part = 0; part < 2; part++) {  // fluid neighbours, then boundary ones
        if (part == 1 && !gfluid) break;
        const int lo = (int)cstart[part * cap1 + u0];
        const int hi = (int)cstart[part * cap1 + u1];
        const bool mine = reach && (part == 0 || afluid);
        const bool ddt = ddt_on && part == 0;
#pragma unroll 1
        for (int base = lo; base < hi; base += 32) {
          const int j = base + lane;
          if (j < hi) {
            t_pos[wb + lane] = posc[j];
            t_vel[wb + lane] = velrho[j];
            t_q[wb + lane] = press[j];
          }
          __syncwarp();
          const int nk = min(32, hi - base);
          if (mine) {
#pragma unroll 2
            for (int k = 0; k < nk; k++) {
              const float4 pb = t_pos[wb + k];
              const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
              const float ry = sy - pb.y, rz = sz - pb.z;
              const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
              if (__float_as_uint(r2) - 1u < r2max_u) {
                const float4 vb = t_vel[wb + k];
                if (afluid) {
                  pair_fluid(va, Pa, kv, hih, eta2, rx, ry, rz, r2, vb, t_q[wb + k], ddt, A);
                  if (part) A.cntb++; else A.cnt++;
                } else {
                  pair_boundary(va, hih, rx, ry, rz, r2, vb, A);
                  A.cnt++;
                }
              }
            }
          }
          __syncwarp();
        }
      }
    }
  }
  finish_target(C, i, n, cidx, has, afluid, va, A, want_dt, ace, mu_out, dyn);
}

// tau/rho of Eq 25 from the sums g of V_b-weighted velocity differences
// (units of 1/(m cw)): S, |S| = (2 S:S)^(1/2) / 2, nu_SPS = (C_S Delta)^2 |S|.
__device__ __forceinline__ void sps_tau_from_gradient(const CaseConst &C, float gxx, float gyy,
                                                      float gzz, float gxy, float gxz,
                                                      float gyz, float4 &t4, float2 &t2) {
  const float k = C.m * C.cw;
  const float sxx = k * gxx, syy = k * gyy, szz = k * gzz;
  const float sxy = 0.5f * k * gxy, sxz = 0.5f * k * gxz, syz = 0.5f * k * gyz;
  const float ss = fmaf(sxx, sxx, fmaf(syy, syy, szz * szz)) +
                   2.f * fmaf(sxy, sxy, fmaf(sxz, sxz, syz * syz));
  const float smag = 0.5f * sqrtf(2.f * ss);
  const float nu2 = 2.f * C.sps_cs2 * smag;
  const float tr3 = (sxx + syy + szz) * (1.f / 3.f);
  const float iso = -(2.f / 3.f) * C.sps_cl2 * smag * smag;
  t4 = make_float4(fmaf(nu2, sxx - tr3, iso), fmaf(nu2, syy - tr3, iso),
                   fmaf(nu2, szz - tr3, iso), nu2 * sxy);
  t2 = make_float2(nu2 * sxz, nu2 * syz);
}

// First neighbour pass of the laminar + SPS model (Eq 24-25): for every
// fluid particle a of a case with visc_mode 1, the SPH velocity gradient
// G^{ij} = sum_{b in P} V_b (v_b - v_a)^i grad^j_a W_ab, its symmetric part
// S, |S| = (2 S:S)^(1/2) / 2 and nu_SPS = (C_S Delta)^2 |S|, then
//   tau/rho = 2 nu_SPS (S - tr(S)/3 I) - (2/3) C_l Delta^2 |S|^2 I,
// written as tau4 = (xx, yy, zz, xy), tau2 = (xz, yz); zero for the others.
// Same rows, pruning and 32-candidate test as the interaction kernel.
template <int M>
__global__ void __launch_bounds__(128, 6)
k_strain(int n, const int *__restrict__ nvalid_p, const uint32_t *__restrict__ keys,
         const float4 *__restrict__ posc, const float4 *__restrict__ velrho,
         const uint16_t *__restrict__ cid, const uint32_t *__restrict__ cstart, uint32_t cap1,
         int nbits, const CaseConst *__restrict__ cc, float4 *__restrict__ tau4,
         float2 *__restrict__ tau2) {
  const unsigned full = 0xffffffffu;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nvalid = *nvalid_p;
  const bool has = i < nvalid;
  const int cidx = i < n ? (int)cid[i] : 0;
  const CaseConst &C = cc[cidx];
  const uint32_t key = has ? keys[i] : 0u;
  const bool act = has && !key_boundary(key, nbits) && C.visc == 1;
  if (__all_sync(full, !act)) {
    if (i < n) {
      tau4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      tau2[i] = make_float2(0.f, 0.f);
    }
    return;
  }
  const int gc = (int)key_cell(key, nbits);
  const int nx = C.nx, nxy = C.nx * C.ny;
  const float cs = C.csf, ics = C.inv_csf, r2max = C.r2max, hih = C.half_inv_h;
  const float r2prune = r2max * 1.0001f;
  const unsigned r2max_u = __float_as_uint(r2max) - 1u;
  const float4 pa = act ? posc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 va = act ? velrho[i] : make_float4(0.f, 0.f, 0.f, 1.f);
  float gxx = 0.f, gyy = 0.f, gzz = 0.f, gxy = 0.f, gxz = 0.f, gyz = 0.f;
  constexpr int W = 2 * M + 1;
#pragma unroll 1
  for (int row = 0; row < W * W; row++) {
    const int dy = row % W - M, dz = row / W - M;
    const float gy = slab_gap(dy, pa.y, cs), gz = slab_gap(dz, pa.z, cs);
    const float d2 = fmaf(gy, gy, gz * gz);
    int loF = 0, hiF = 0, loB = 0, hiB = 0;
    if (act && d2 < r2prune) {
      const float L = sqrtf(r2prune - d2);
      const int kx0 = max(-M, (int)floorf((pa.x - L) * ics));
      const int kx1 = min(M, (int)floorf((pa.x + L) * ics));
      const int c0 = gc + dz * nxy + dy * nx + kx0;
      const int c1 = gc + dz * nxy + dy * nx + kx1 + 1;
      loF = (int)cstart[c0];
      hiF = (int)cstart[c1];
      loB = (int)cstart[cap1 + c0];
      hiB = (int)cstart[cap1 + c1];
    }
    const float sy = fmaf(-(float)dy, cs, pa.y), sz = fmaf(-(float)dz, cs, pa.z);
#pragma unroll 1
    for (int part = 0; part < 2; part++) {  // b in F, then b in B
      const int lo = part ? loB : loF;
      const int len = (part ? hiB : hiF) - lo;
      const int maxlen = (int)__reduce_max_sync(full, (unsigned)max(len, 0));
#pragma unroll 1
      for (int base = 0; base < maxlen; base += 32) {
        unsigned m = 0u;
        const int nk = min(32, maxlen - base);
#pragma unroll 8
        for (int k = 0; k < nk; k++) {
          if (base + k < len) {
            const float4 pb = posc[lo + base + k];
            const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
            const float ry = sy - pb.y, rz = sz - pb.z;
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            if (__float_as_uint(r2) - 1u < r2max_u) m |= 1u << k;
          }
        }
        while (__any_sync(full, m != 0u)) {
          if (m) {
            const int k = 31 - __clz(m);
            m ^= 1u << k;
            const int j = lo + base + k;
            const float4 pb = posc[j];
            const float4 vb = velrho[j];
            const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
            const float ry = sy - pb.y, rz = sz - pb.z;
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            const float t = fmaf(-hih, r2 * rsqrtf(r2), 1.f);
            const float w = t * t * t * __fdividef(1.f, vb.w);  // V_b grad W / (m cw r_ab)
            const float dvx = vb.x - va.x, dvy = vb.y - va.y, dvz = vb.z - va.z;
            gxx = fmaf(w * dvx, rx, gxx);
            gyy = fmaf(w * dvy, ry, gyy);
            gzz = fmaf(w * dvz, rz, gzz);
            gxy = fmaf(w, fmaf(dvx, ry, dvy * rx), gxy);
            gxz = fmaf(w, fmaf(dvx, rz, dvz * rx), gxz);
            gyz = fmaf(w, fmaf(dvy, rz, dvz * ry), gyz);
          }
        }
      }
    }
  }
  if (i >= n) return;
  if (!act) {
    tau4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    tau2[i] = make_float2(0.f, 0.f);
    return;
  }
  sps_tau_from_gradient(C, gxx, gyy, gzz, gxy, gxz, gyz, tau4[i], tau2[i]);
}

// ---- modified dynamic boundary condition (Eq 38-39) ------------------------------

// Solves A x = b (4x4, FP64) by Gaussian elimination with partial pivoting;
// returns det(A); x is left unset when det == 0.
__device__ double solve4(double A[4][4], double b[4], double x[4]) {
  double det = 1.0;
#pragma unroll
  for (int c = 0; c < 4; c++) {
    int piv = c;
#pragma unroll
    for (int r = c + 1; r < 4; r++)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (A[piv][c] == 0.0) return 0.0;
    if (piv != c) {
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const double t = A[c][k];
        A[c][k] = A[piv][k];
        A[piv][k] = t;
      }
      const double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
      det = -det;
    }
    det *= A[c][c];
#pragma unroll
    for (int r = c + 1; r < 4; r++) {
      const double f = A[r][c] / A[c][c];
#pragma unroll
      for (int k = c; k < 4; k++) A[r][k] -= f * A[c][k];
      b[r] -= f * b[c];
    }
  }
#pragma unroll
  for (int r = 3; r >= 0; r--) {
    double v = b[r];
#pragma unroll
    for (int k = r + 1; k < 4; k++) v -= A[r][k] * x[k];
    x[r] = v / A[r][r];
  }
  return det;
}

constexpr double kMdbcDetMin = 1e-3;  // |det| below: Shepard value, zero gradient

// One thread per particle (sorted order); boundary particles of mDBC cases
// get their density from the ghost node r_G = r_B + ghost (Eq 38) and, with
// mdbc_slip, their velocity from the Shepard sum of Eq 39.  The moment sums
// run over fluid particles within 2h of r_G, found from the ghost's own cell
// (rows clamped to the grid).  stage selects the time of the imposed wall
// velocity: t (0) or t + dt/2 (1).  Also refreshes P/rho of the particle.
// LIST: the state is in the cells of a neighbour list's build, particles up
// to half the skin outside them, so the rows reach M + 1 cells and prune at
// 2h + skin/2.
template <int M, bool LIST>
__global__ void __launch_bounds__(128)
k_mdbc(int n, const int *__restrict__ nvalid_p, const uint32_t *__restrict__ keys, State st,
       float *__restrict__ press, const uint32_t *__restrict__ cstart, int nbits,
       const CaseConst *__restrict__ cc, const CaseDyn *__restrict__ dyn, int stage) {
  const unsigned full = 0xffffffffu;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nvalid = *nvalid_p;
  const bool has = i < nvalid;
  const int cidx = i < n ? (int)st.cid[i] : 0;
  const CaseConst &C = cc[cidx];
  const uint32_t key = has ? keys[i] : 0u;
  const bool act = has && key_boundary(key, nbits) && C.bmode == 1;
  if (__all_sync(full, !act)) return;
  const float cs = C.csf, ics = C.inv_csf, r2max = C.r2max, hih = C.half_inv_h;
  float r2prune = r2max * 1.0001f;
  if (LIST) {
    const float R = sqrtf(r2max) + 0.5f * dyn[cidx].skin;
    r2prune = R * R * 1.0001f;
  }
  constexpr int MR = LIST ? M + 1 : M;
  // ghost position: cell of B shifted by the whole cells of (offset + ghost)
  int cx = 0, cy = 0, cz = 0;
  float4 pb = make_float4(0.f, 0.f, 0.f, 0.f), g = pb;
  if (act) {
    decode_cell(key_cell(key, nbits) - C.cellbase, C.nx, C.ny, cx, cy, cz);
    pb = st.posc[i];
    g = st.ghost[i];
  }
  const float qx0 = pb.x + g.x, qy0 = pb.y + g.y, qz0 = pb.z + g.z;
  const int sx = (int)floorf(qx0 * ics), sy = (int)floorf(qy0 * ics), sz = (int)floorf(qz0 * ics);
  const int gx = cx + sx, gy = cy + sy, gz = cz + sz;                       // ghost cell
  const float ox = fmaf(-(float)sx, cs, qx0), oy = fmaf(-(float)sy, cs, qy0),
              oz = fmaf(-(float)sz, cs, qz0);                               // offset in it
  const int nx = C.nx, ny = C.ny, nz = C.nz, nxy = nx * ny;
  const int base0 = (int)C.cellbase;
  // moment sums (per unit particle mass): A00 = sum W / rho_b, A0k = sum e_k W / rho_b,
  // Ak0 = sum F d_k / rho_b, Akl = sum F d_k e_l / rho_b (e = -d = r_b - r_G),
  // vs = sum v W / rho_b, and the right-hand side for (rho_G - rho0, grad rho_G):
  // r0 = sum W (rho_b - rho0) / rho_b, rk = sum F d_k (rho_b - rho0) / rho_b.  The
  // same system as for rho_G itself (A (rho0, 0) is rho0 times A's first column),
  // but its right-hand side has no FP32 cancellation of rho0-sized terms.
  float a00 = 0.f, a01 = 0.f, a02 = 0.f, a03 = 0.f, a10 = 0.f, a20 = 0.f, a30 = 0.f;
  float dxx = 0.f, dyy = 0.f, dzz = 0.f, dxy = 0.f, dxz = 0.f, dyz = 0.f;
  float r0 = 0.f, r1 = 0.f, r2s = 0.f, r3 = 0.f, vsx = 0.f, vsy = 0.f, vsz = 0.f;
  constexpr int W = 2 * MR + 1;
#pragma unroll 1
  for (int row = 0; row < W * W; row++) {
    const int dy = row % W - MR, dz = row / W - MR;
    const int yy = gy + dy, zz = gz + dz;
    int lo = 0, hi = 0;
    const float sgy = slab_gap(dy, oy, cs), sgz = slab_gap(dz, oz, cs);
    const float d2 = fmaf(sgy, sgy, sgz * sgz);
    if (act && d2 < r2prune && yy >= 0 && yy < ny && zz >= 0 && zz < nz) {
      const float L = sqrtf(r2prune - d2);
      const int x0 = max(0, gx + max(-MR, (int)floorf((ox - L) * ics)));
      const int x1 = min(nx - 1, gx + min(MR, (int)floorf((ox + L) * ics)));
      if (x1 >= x0) {
        const int c0 = base0 + zz * nxy + yy * nx;
        lo = (int)cstart[c0 + x0];  // fluid segment only (b in F)
        hi = (int)cstart[c0 + x1 + 1];
      }
    }
    const float ry0 = fmaf((float)(gy - yy), cs, oy), rz0 = fmaf((float)(gz - zz), cs, oz);
    const int len = hi - lo;
    const int maxlen = (int)__reduce_max_sync(full, (unsigned)max(len, 0));
#pragma unroll 1
    for (int k = 0; k < maxlen; k++) {
      if (k < len) {
        const int j = lo + k;
        const float4 pf = st.posc[j];
        const float ddx = fmaf((float)gx - pf.w, cs, ox - pf.x);  // d = r_G - r_b
        const float ddy = ry0 - pf.y, ddz = rz0 - pf.z;
        const float rr2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
        if (rr2 < r2max) {
          const float4 vb = st.velrho[j];
          const float ib = __fdividef(1.f, vb.w);
          const float t = fmaf(-hih, rr2 * rsqrtf(rr2 + 1e-30f), 1.f);
          const float t3 = t * t * t;
          const float w = C.wk * t3 * t * fmaf(-4.f, t, 5.f);  // W (Eq 11)
          const float f = C.cw * t3;                            // grad_G W = f d
          const float wv = w * ib, fv = f * ib;
          const float dr = (vb.w - C.rho0) * ib;  // (rho_b - rho0) / rho_b
          a00 += wv;
          a01 = fmaf(-wv, ddx, a01);
          a02 = fmaf(-wv, ddy, a02);
          a03 = fmaf(-wv, ddz, a03);
          a10 = fmaf(fv, ddx, a10);
          a20 = fmaf(fv, ddy, a20);
          a30 = fmaf(fv, ddz, a30);
          dxx = fmaf(fv * ddx, ddx, dxx);
          dyy = fmaf(fv * ddy, ddy, dyy);
          dzz = fmaf(fv * ddz, ddz, dzz);
          dxy = fmaf(fv * ddx, ddy, dxy);
          dxz = fmaf(fv * ddx, ddz, dxz);
          dyz = fmaf(fv * ddy, ddz, dyz);
          r0 = fmaf(w, dr, r0);
          r1 = fmaf(f * dr, ddx, r1);
          r2s = fmaf(f * dr, ddy, r2s);
          r3 = fmaf(f * dr, ddz, r3);
          vsx = fmaf(wv, vb.x, vsx);
          vsy = fmaf(wv, vb.y, vsy);
          vsz = fmaf(wv, vb.z, vsz);
        }
      }
    }
  }
  if (!act) return;
  // imposed velocity of B at the evaluation time (Eq 37)
  float vw[3] = {0.f, 0.f, 0.f};
  const uint8_t code = st.code[i];
  if (code >= 2) {
    const int gi = code - 2;
    const CaseDyn &D = dyn[cidx];
    const double te = D.t + (stage ? 0.5 * D.dt : 0.0);
    const float v = (float)(C.mot_amp[gi] * C.mot_omega[gi] *
                            cos(C.mot_omega[gi] * te + C.mot_phase[gi]));
    vw[0] = v * C.mot_axis[gi][0];
    vw[1] = v * C.mot_axis[gi][1];
    vw[2] = v * C.mot_axis[gi][2];
  }
  float4 out = st.velrho[i];
  if (!(a00 > 0.f)) {  // no fluid near the ghost
    out.w = C.rho0;
    if (C.mdbc_slip) {
      out.x = vw[0];
      out.y = vw[1];
      out.z = vw[2];
    }
  } else {
    double A[4][4] = {{a00, a01, a02, a03},
                      {a10, -dxx, -dxy, -dxz},
                      {a20, -dxy, -dyy, -dyz},
                      {a30, -dxz, -dyz, -dzz}};
    double b[4] = {r0, r1, r2s, r3}, x[4] = {0.0, 0.0, 0.0, 0.0};
    // the sums are per unit particle mass: the determinant of the moment
    // matrix with volumes V_b = m / rho_b is m^4 times this one
    const double m2 = C.m_d * C.m_d;
    const double det = solve4(A, b, x) * (m2 * m2);
    const double shep = (double)C.rho0 + (double)r0 / (double)a00;  // Shepard value
    double rhoB = shep;
    if (fabs(det) >= kMdbcDetMin) {
      // Eq 38 with r_B - r_G = -ghost
      rhoB = (double)C.rho0 + x[0] - ((double)g.x * x[1] + (double)g.y * x[2] + (double)g.z * x[3]);
      if (!(rhoB > 0.0 && rhoB < 1e30)) rhoB = shep;  // not a usable density
    }
    out.w = (float)rhoB;
    const float vgx = vsx / a00, vgy = vsy / a00, vgz = vsz / a00;  // Eq 39
    if (C.mdbc_slip == 1) {
      out.x = 2.f * vw[0] - vgx;
      out.y = 2.f * vw[1] - vgy;
      out.z = 2.f * vw[2] - vgz;
    } else if (C.mdbc_slip == 2) {
      const float gn = sqrtf(g.x * g.x + g.y * g.y + g.z * g.z);
      const float inv = gn > 0.f ? 1.f / gn : 0.f;
      const float nx_ = g.x * inv, ny_ = g.y * inv, nz_ = g.z * inv;
      const float vn = vgx * nx_ + vgy * ny_ + vgz * nz_;
      const float wn = vw[0] * nx_ + vw[1] * ny_ + vw[2] * nz_;
      const float k2 = 2.f * (wn - vn);
      out.x = fmaf(k2, nx_, vgx);
      out.y = fmaf(k2, ny_, vgy);
      out.z = fmaf(k2, nz_, vgz);
    }
  }
  st.velrho[i] = out;
  press[i] = tait_pressure(C, out.w) / out.w;
}

// ---- time step and motion ----------------------------------------------------

__device__ __forceinline__ double motion_disp(const CaseConst &C, int g, double t) {
  return C.mot_amp[g] * (sin(C.mot_omega[g] * t + C.mot_phase[g]) - sin(C.mot_phase[g]));
}
__device__ __forceinline__ double motion_vel(const CaseConst &C, int g, double t) {
  return C.mot_amp[g] * C.mot_omega[g] * cos(C.mot_omega[g] * t + C.mot_phase[g]);
}

__global__ void k_dt(int ncases, const CaseConst *__restrict__ cc, CaseDyn *__restrict__ dyn) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncases) return;
  const CaseConst &C = cc[c];
  CaseDyn &D = dyn[c];
  if (!C.active) return;
  unsigned bits = D.dtmin_bits;
  double dt;
  if (C.dt_fixed > 0.0) {
    dt = C.dt_fixed;
  } else if (bits >= kFloatInfBits) {
    dt = C.cfl * C.h_d / C.cs0_d;  // no fluid: dt_f = inf, dt_cv = h / cs0
  } else {
    dt = C.cfl * (double)__uint_as_float(bits);
  }
  if (dt < C.dt_min) D.flags |= kFlagDtMin;
  if (C.t_end > 0.0 && D.t >= C.t_end) dt = 0.0;  // finished cases stay put
  D.dt = dt;
  D.dtmin_bits = kFloatInfBits;
  for (int g = 0; g < C.nmot; g++) {
    double d0 = motion_disp(C, g, D.t);
    D.mot[g][0] = motion_disp(C, g, D.t + 0.5 * dt) - d0;
    D.mot[g][1] = motion_vel(C, g, D.t + 0.5 * dt);
    D.mot[g][2] = motion_disp(C, g, D.t + dt) - d0;
    D.mot[g][3] = motion_vel(C, g, D.t + dt);
  }
}

__global__ void k_end_step(int ncases, const CaseConst *__restrict__ cc,
                           CaseDyn *__restrict__ dyn) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncases || !cc[c].active) return;
  CaseDyn &D = dyn[c];
  if (D.dt > 0.0) {
    D.t += D.dt;
    D.step += 1;
  }
  D.v2max_bits = 0u;
}

// ---- Symplectic predictor / corrector ------------------------------------------

// Moves a particle by disp (FP64, per axis) from the cell of key k; returns
// the new key (or key_out) and writes the new offsets.
__device__ __forceinline__ uint32_t move_particle(uint32_t k, const float4 &p, const double disp[3],
                                                  const CaseConst &C, bool boundary, int nbits,
                                                  float4 &pout, bool &left) {
  int cx, cy, cz;
  decode_cell(key_cell(k, nbits) - C.cellbase, C.nx, C.ny, cx, cy, cz);
  float ox, oy, oz;
  cx += shift_axis(p.x, disp[0], C, ox);
  cy += shift_axis(p.y, disp[1], C, oy);
  cz += shift_axis(p.z, disp[2], C, oz);
  const int M = C.margin;
  left = !(cx >= M && cx < C.nx - M && cy >= M && cy < C.ny - M && cz >= M && cz < C.nz - M);
  if (left) {
    // frozen: keep a float position relative to the grid origin
    pout = make_float4((float)(cx * C.cs + ox), (float)(cy * C.cs + oy),
                       (float)(cz * C.cs + oz), 0.f);
    return key_out(nbits);
  }
  pout = make_float4(ox, oy, oz, (float)cx);
  uint32_t lin = ((uint32_t)cz * C.ny + cy) * C.nx + cx;
  return key_make(C.cellbase + lin, boundary, nbits);
}

// Eq 33-34 half step of one particle: displacement dt/2 v^n (FP64) and
// v, rho at n+1/2; boundary particles: density only (clamped), moving ones
// displaced by Eq 37 at t + dt/2.
__device__ __forceinline__ void predictor_core(const CaseConst &C, const CaseDyn &D,
                                               uint8_t code, const float4 &v, const float4 &a,
                                               double disp[3], float4 &vn) {
  const double hdt = 0.5 * D.dt;
  const float hdtf = (float)hdt;
  if (code == 0) {
    disp[0] = hdt * (double)v.x;
    disp[1] = hdt * (double)v.y;
    disp[2] = hdt * (double)v.z;
    vn = make_float4(fmaf(hdtf, a.x, v.x), fmaf(hdtf, a.y, v.y), fmaf(hdtf, a.z, v.z),
                     fmaf(hdtf, a.w, v.w));
  } else {
    float rho = fmaf(hdtf, a.w, v.w);
    if (C.clamp && rho < C.rho0) rho = C.rho0;
    if (code >= 2) {
      const int g = code - 2;
      const double d = D.mot[g][0];
      const float vm = (float)D.mot[g][1];
      disp[0] = d * C.mot_axis[g][0];
      disp[1] = d * C.mot_axis[g][1];
      disp[2] = d * C.mot_axis[g][2];
      vn = make_float4(vm * C.mot_axis[g][0], vm * C.mot_axis[g][1], vm * C.mot_axis[g][2], rho);
    } else {
      disp[0] = disp[1] = disp[2] = 0.0;
      vn = make_float4(v.x, v.y, v.z, rho);
    }
  }
}

__global__ void k_predictor(int n, const uint32_t *__restrict__ keys_in, State src,
                            const float4 *__restrict__ ace, const CaseConst *__restrict__ cc,
                            CaseDyn *__restrict__ dyn, int nbits, float4 *__restrict__ posc_out,
                            float4 *__restrict__ velrho_out, uint32_t *__restrict__ keys_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys_in[i];
  const float4 p = src.posc[i];
  const float4 v = src.velrho[i];
  if (k >= key_out(nbits)) {  // frozen or released: unchanged
    posc_out[i] = p;
    velrho_out[i] = v;
    keys_out[i] = k;
    return;
  }
  const int cidx = src.cid[i];
  const uint8_t code = src.code[i];
  const CaseConst &C = cc[cidx];
  const CaseDyn &D = dyn[cidx];
  double disp[3];
  float4 vn;
  predictor_core(C, D, code, v, ace[i], disp, vn);
  float4 pn;
  bool left;
  uint32_t kn = move_particle(k, p, disp, C, code != 0, nbits, pn, left);
  if (left) {
    // left the domain at the half step: frozen at state n
    int cx, cy, cz;
    decode_cell(key_cell(k, nbits) - C.cellbase, C.nx, C.ny, cx, cy, cz);
    pn = make_float4((float)(cx * C.cs + p.x), (float)(cy * C.cs + p.y),
                     (float)(cz * C.cs + p.z), 0.f);
    vn = v;
    atomicAdd(&dyn[cidx].n_out, 1);
  }
  posc_out[i] = pn;
  velrho_out[i] = vn;
  keys_out[i] = kn;
}

// Eq 33-34 full step of one particle from state n (key k, pn, vn), the
// half-step density rhoh and F, R at n+1/2 (a): the new position (cell +
// offset, FP64 displacement), velocity and density; returns the new key.
__device__ __forceinline__ uint32_t corrector_core(const CaseConst &C, const CaseDyn &D,
                                                   uint8_t code, uint32_t k, const float4 &pn,
                                                   const float4 &vn, float rhoh, const float4 &a,
                                                   int nbits, int cidx, CaseDyn *dyn,
                                                   float4 &pnew, float4 &vnew,
                                                   double *disp_out = nullptr) {
  const double dt = D.dt;
  const float dtf = (float)dt;
  // Eq 34: rho^{n+1} = rho^n (2 - eps) / (2 + eps), eps = -(R / rho^{n+1/2}) dt
  const float eps = -(a.w / rhoh) * dtf;
  float rho = vn.w * (2.f - eps) / (2.f + eps);
  double disp[3];
  if (code == 0) {
    vnew = make_float4(fmaf(dtf, a.x, vn.x), fmaf(dtf, a.y, vn.y), fmaf(dtf, a.z, vn.z), rho);
    // r^{n+1} = r^n + dt (v^{n+1} + v^n) / 2: the FP32 sum of two FP32
    // velocities is exact to within one rounding; dt multiplies in FP64
    const double hdt = 0.5 * dt;
    disp[0] = hdt * (double)(vnew.x + vn.x);
    disp[1] = hdt * (double)(vnew.y + vn.y);
    disp[2] = hdt * (double)(vnew.z + vn.z);
  } else {
    if (C.clamp && rho < C.rho0) rho = C.rho0;
    if (code >= 2) {
      const int g = code - 2;
      const double d = D.mot[g][2];
      const float vm = (float)D.mot[g][3];
      disp[0] = d * C.mot_axis[g][0];
      disp[1] = d * C.mot_axis[g][1];
      disp[2] = d * C.mot_axis[g][2];
      vnew = make_float4(vm * C.mot_axis[g][0], vm * C.mot_axis[g][1], vm * C.mot_axis[g][2],
                         rho);
    } else {
      disp[0] = disp[1] = disp[2] = 0.0;
      vnew = make_float4(vn.x, vn.y, vn.z, rho);
    }
  }
  if (disp_out) {
    disp_out[0] = disp[0];
    disp_out[1] = disp[1];
    disp_out[2] = disp[2];
  }
  bool left;
  const uint32_t kn = move_particle(k, pn, disp, C, code != 0, nbits, pnew, left);
  if (left) atomicAdd(&dyn[cidx].n_out, 1);  // frozen at state n+1
  return kn;
}

__global__ void k_corrector(int n, const uint32_t *__restrict__ perm2,
                            const uint32_t *__restrict__ keys_half,
                            const uint32_t *__restrict__ keys_n, State sn, State x,
                            const float4 *__restrict__ ace, const CaseConst *__restrict__ cc,
                            CaseDyn *__restrict__ dyn, int nbits,
                            uint32_t *__restrict__ keys_next) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t p = perm2[i];
  const uint32_t kh = keys_half[i];
  if (kh >= key_out(nbits)) {  // frozen (already in x) or released
    keys_next[i] = kh;
    return;
  }
  const float4 pn = sn.posc[p];
  const float4 vn = sn.velrho[p];
  const uint32_t k = keys_n[p];
  const int cidx = x.cid[i];
  const uint8_t code = x.code[i];
  const CaseConst &C = cc[cidx];
  const CaseDyn &D = dyn[cidx];
  float4 pnew, vnew;
  const uint32_t kn = corrector_core(C, D, code, k, pn, vn, x.velrho[i].w, ace[i], nbits, cidx,
                                     dyn, pnew, vnew);
  x.posc[i] = pnew;
  x.velrho[i] = vnew;
  keys_next[i] = kn;
}

// ---- neighbour lists (pi_variant 3-5) ---------------------------------------------
//
// The Symplectic step evaluates the interaction on state n and on state n+1/2.
// Instead of sorting again for n+1/2, the candidate test runs on state n with
// radius 2h + skin and writes every chunk of candidates that passes as a
// record (first index | row code, mask) into a per-target list; both
// evaluations walk the records and keep the pairs with 0 < r^2 < (2h)^2 at
// their own state.  The half-step state keeps the cells of state n (offsets
// may leave [0, cs) by a half-step displacement), so relative positions stay
// cell + offset in FP32.  The skin covers twice the largest displacement since
// the build, which the predictor checks (kFlagSkin).  Variants 3 and 4 build
// the list every step; 5 keeps it, with the particle order and cells, until a
// particle of the case could leave the skin.  The pair set of each evaluation
// is the same as with a fresh neighbour list; only the order of the sums
// differs.


// The interaction over a target's list (state n or n+1/2, same order and
// cells): the pair terms of k_interact for the entries inside 2h.  EXT 1
// adds the Eq 19-20 density diffusion, EXT 2 also laminar + SPS (tau4/tau2
// from k_strain_list), for the cases that use them.
// Arguments of the interaction over the neighbour list (one struct, so that
// the one-target body below serves both launch forms).
struct ListArgs {
  int n;
  const int *nvalid_p;
  const uint32_t *keys;
  const float4 *posc, *velrho;
  const float *press;
  const uint16_t *cid;
  const uint32_t *cstart;
  uint32_t cap1;
  int nbits;
  const CaseConst *cc;
  CaseDyn *dyn;
  float4 *ace;
  int want_dt;
  const uint2 *list;
  int cap;  // records per target: record r of target i at list[i cap + r]
  const uint16_t *count;
  const float4 *tau4;
  const float2 *tau2;
  float *mu_out;
  // wide records (beyond 2^25 particles): the keys of the build's cells,
  // whose cell gives a record's row (valid for every candidate of a kept
  // list, also where a particle left at the half step)
  const uint32_t *row_keys;
};

// One target i of the list walk (all 32 lanes of the warp call it together).
// G lanes share a target (G = 1, 2, 4 or 8; sub = the lane's rank among
// them): lane sub takes the candidates of each record at the bit positions
// sub, sub + G, sub + 2G, ..., so the lanes of a target load neighbouring
// candidates together (fewer L1 wavefronts per gather), and the G partial
// sums are combined by a butterfly over the G lanes at the end.
template <int EXT, int G, int W = 0>
__device__ __forceinline__ void list_target(const int i, const int sub, const ListArgs &a) {
  const unsigned full = 0xffffffffu;
  const int n = a.n;
  const int *__restrict__ nvalid_p = a.nvalid_p;
  const uint32_t *__restrict__ keys = a.keys;
  const float4 *__restrict__ posc = a.posc;
  const float4 *__restrict__ velrho = a.velrho;
  const float *__restrict__ press = a.press;
  const uint16_t *__restrict__ cid = a.cid;
  const uint32_t *__restrict__ cstart = a.cstart;
  const uint32_t cap1 = a.cap1;
  const int nbits = a.nbits;
  const CaseConst *__restrict__ cc = a.cc;
  CaseDyn *__restrict__ dyn = a.dyn;
  float4 *__restrict__ ace = a.ace;
  const int want_dt = a.want_dt;
  const uint2 *__restrict__ list = a.list;
  const int cap = a.cap;
  const uint16_t *__restrict__ count = a.count;
  const float4 *__restrict__ tau4 = a.tau4;
  const float2 *__restrict__ tau2 = a.tau2;
  float *__restrict__ mu_out = a.mu_out;
  const int nvalid = *nvalid_p;
  const uint32_t key = i < nvalid ? keys[i] : key_out(nbits);
  const bool has = key < key_out(nbits);  // not frozen at this state
  const int cidx = i < n ? (int)cid[i] : 0;
  const CaseConst &C = cc[cidx];
  const bool afluid = has && !key_boundary(key, nbits);
  const float cs = C.csf, eta2 = C.eta2, hih = C.half_inv_h;
  const unsigned r2max_u = __float_as_uint(C.r2max) - 1u;
  const float4 pa = has ? posc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 va = has ? velrho[i] : make_float4(0.f, 0.f, 0.f, 1.f);
  const float Pa = has ? press[i] * va.w : 0.f;
  const float kv = C.kvisc * va.w;
  const bool ddt_on = C.ddt != 0;
  Ext X;
  X.C = &C;
  X.hyd = EXT >= 1 && C.ddt == 2;
  X.sps = EXT == 2 && C.visc == 1 && afluid;
  X.kl = -4.f * C.nu0 * va.w;
  X.tau4 = tau4;
  X.tau2 = tau2;
  {
    const float4 t4 = X.sps ? tau4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 t2 = X.sps ? tau2[i] : make_float2(0.f, 0.f);
    X.ta[0] = va.w * t4.x;
    X.ta[1] = va.w * t4.y;
    X.ta[2] = va.w * t4.z;
    X.ta[3] = va.w * t4.w;
    X.ta[4] = va.w * t2.x;
    X.ta[5] = va.w * t2.y;
  }
  const int jb = (int)cstart[cap1 - 1];  // first boundary particle of the key order
  const int nrec = has ? (int)count[i] : 0;
  const bool warp_fluid = __all_sync(full, afluid || !has);
  Acc A = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u};
  const uint2 *__restrict__ mine = list + (int64_t)i * cap;
  // two candidates per lane per iteration (their loads issued together),
  // records taken in order: the warp waits only for its lane with the most
  // candidates in total
  int r = 0;
  unsigned cm = 0u;
  int cbase = 0;
  float sy = 0.f, sz = 0.f;
  // the next record of the lane: base index, candidate mask, row offsets
  // the lane's bit positions within a record
  const unsigned sel = (G == 1 ? 0xffffffffu : G == 2 ? 0x55555555u : G == 4 ? 0x11111111u
                                                                    : 0x01010101u) << sub;
  // wide records: the rows relative to the target's own cell
  int tcy = 0, tcz = 0;
  if (W && nrec) {
    int tcx;
    decode_cell(key_cell(a.row_keys[i], nbits) - C.cellbase, C.nx, C.ny, tcx, tcy, tcz);
  }
  auto next_record = [&]() {
    const uint2 rec = mine[r++];
    int rdy, rdz;
    if (W) {
      cbase = (int)rec.x;
      int bx, by, bz;
      decode_cell(key_cell(a.row_keys[cbase], nbits) - C.cellbase, C.nx, C.ny, bx, by, bz);
      rdy = by - tcy;
      rdz = bz - tcz;
    } else {
      cbase = (int)(rec.x & kListIndexMask);
      list_row_decode(rec.x, rdy, rdz);
    }
    cm = rec.y & sel;
    sy = fmaf(-(float)rdy, cs, pa.y);
    sz = fmaf(-(float)rdz, cs, pa.z);
  };
#pragma unroll 1
  for (;;) {
    // (a record holds at least one candidate, but with G > 1 maybe none of
    // this lane's)
    if (G == 1) {
      if (cm == 0u && r < nrec) next_record();
    } else {
      while (cm == 0u && r < nrec) next_record();
    }
    if (!__any_sync(full, cm != 0u)) break;
    if (cm) {
      // the lane's next two candidates in list order; the second may open the
      // next record, so no slot idles at the end of an odd record
      const int k1 = 31 - __clz(cm);
      cm ^= 1u << k1;
      const int j1 = cbase + k1;
      const float sy1 = sy, sz1 = sz;
      if (G == 1) {
        if (cm == 0u && r < nrec) next_record();
      } else {
        while (cm == 0u && r < nrec) next_record();
      }
      const bool h2 = cm != 0u;
      const int k2 = h2 ? 31 - __clz(cm) : k1;
      if (h2) cm ^= 1u << k2;
      const int j2 = h2 ? cbase + k2 : j1;
      const float4 pb1 = posc[j1];
      const float4 pb2 = posc[j2];
      const float4 vb1 = velrho[j1];
      const float4 vb2 = velrho[j2];
      const float q1 = press[j1], q2 = press[j2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const float4 pb = u ? pb2 : pb1;
        const float4 vb = u ? vb2 : vb1;
        const int j = u ? j2 : j1;
        const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
        const float ry = (u ? sy : sy1) - pb.y, rz = (u ? sz : sz1) - pb.z;
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        if ((u == 0 || h2) && __float_as_uint(r2) - 1u < r2max_u) {
          const bool bfluid = j < jb;
          if (warp_fluid || afluid) {
            pair_fluid<EXT>(va, Pa, kv, hih, eta2, rx, ry, rz, r2, vb, u ? q2 : q1,
                            ddt_on && bfluid, A, &X, j, bfluid);
            if (bfluid) A.cnt++; else A.cntb++;
          } else {
            pair_boundary(va, hih, rx, ry, rz, r2, vb, A);
            A.cnt++;
          }
        }
      }
    }
  }
  if (G > 1) {
    // the G lanes' partial sums; every lane of the target ends with the same
    // totals (each addition is commutative: lanes pair the same operands)
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      A.ax += __shfl_xor_sync(full, A.ax, o);
      A.ay += __shfl_xor_sync(full, A.ay, o);
      A.az += __shfl_xor_sync(full, A.az, o);
      A.s1 += __shfl_xor_sync(full, A.s1, o);
      A.s2 += __shfl_xor_sync(full, A.s2, o);
      A.mur = fmaxf(A.mur, __shfl_xor_sync(full, A.mur, o));
      A.cnt += __shfl_xor_sync(full, A.cnt, o);
      A.cntb += __shfl_xor_sync(full, A.cntb, o);
    }
  }
  finish_target(C, i, n, cidx, has, afluid, va, A, want_dt, ace, mu_out, dyn, sub == 0);
}

// G threads per target, in the key order of the targets (W: wide records).
template <int EXT, int G, int W = 0>
__global__ void __launch_bounds__(EXT == 0 ? 1024 : 128, EXT == 2 ? 6 : (EXT == 0 ? 1 : 0))
k_interact_list(const ListArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  list_target<EXT, G, W>(t / G, t % G, a);
}



// Each pair once (the default physics of Eq 15, 17-18, 21-22 and 36, DBC):
// the momentum term of a pair is antisymmetric, -m cw F r_ab on a and
// +m cw F r_ab on b with F = t^3 [(P_a + P_b)/(rho_a rho_b) + kvisc
// min(v_ab.r_ab, 0)/((r^2 + eta^2)(rho_a + rho_b))], and the continuity
// terms of a and b share t^3 v_ab.r_ab.  A fluid target walks its records
// and takes only the candidates of larger index (in the fluid-first key
// order every boundary particle has a larger index than every fluid one, so
// boundary targets walk nothing); it adds its own terms in registers and the
// partner's with one vector atomic add into sum[b] = (sum_c F_bc r_bc,
// continuity / (m cw)), then its own sums the same way.  The order of the
// atomic additions varies, so the sums are not reproducible bit for bit.
// k_sym_finish turns the sums into dv/dt, drho/dt and the Eq 35 terms.
template <int W>
__global__ void __launch_bounds__(128)
k_interact_sym(const ListArgs a, float4 *__restrict__ sum, unsigned *__restrict__ mu_bits) {
  const unsigned full = 0xffffffffu;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = a.n;
  const int nbits = a.nbits;
  const float4 *__restrict__ posc = a.posc;
  const float4 *__restrict__ velrho = a.velrho;
  const float *__restrict__ press = a.press;
  const int nvalid = *a.nvalid_p;
  const uint32_t key = i < nvalid ? a.keys[i] : key_out(nbits);
  const bool has = key < key_out(nbits);
  const int cidx = i < n ? (int)a.cid[i] : 0;
  const CaseConst &C = a.cc[cidx];
  const bool afluid = has && !key_boundary(key, nbits);
  const float cs = C.csf, eta2 = C.eta2, hih = C.half_inv_h, kvisc = C.kvisc, kddt = C.kddt;
  const unsigned r2max_u = __float_as_uint(C.r2max) - 1u;
  const float4 pa = afluid ? posc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 va = afluid ? velrho[i] : make_float4(0.f, 0.f, 0.f, 1.f);
  const float Qa = afluid ? press[i] : 0.f;  // P_a / rho_a
  const float ia = __fdividef(1.f, va.w);
  const bool ddt_on = C.ddt != 0;
  const int jb = (int)a.cstart[a.cap1 - 1];  // first boundary particle of the key order
  const int nrec = afluid ? (int)a.count[i] : 0;
  const uint2 *__restrict__ mine = a.list + (int64_t)i * a.cap;
  float fx = 0.f, fy = 0.f, fz = 0.f, cont = 0.f, mur = 0.f;
  unsigned nff = 0u, nfb = 0u;
  int r = 0;
  unsigned cm = 0u;
  int cbase = 0;
  float sy = 0.f, sz = 0.f;
  // the next record of the lane, keeping only candidates of index > i
  int tcy = 0, tcz = 0;  // wide records: rows relative to the target's cell
  if (W && nrec) {
    int tcx;
    decode_cell(key_cell(a.row_keys[i], nbits) - C.cellbase, C.nx, C.ny, tcx, tcy, tcz);
  }
  auto next_record = [&]() {
    const uint2 rec = mine[r++];
    cbase = W ? (int)rec.x : (int)(rec.x & kListIndexMask);
    const int lowk = i - cbase + 1;  // first bit of a larger index
    cm = lowk <= 0 ? rec.y : (lowk >= 32 ? 0u : rec.y & (0xffffffffu << lowk));
    int rdy, rdz;
    if (W) {
      int bx, by, bz;
      decode_cell(key_cell(a.row_keys[cbase], nbits) - C.cellbase, C.nx, C.ny, bx, by, bz);
      rdy = by - tcy;
      rdz = bz - tcz;
    } else {
      list_row_decode(rec.x, rdy, rdz);
    }
    sy = fmaf(-(float)rdy, cs, pa.y);
    sz = fmaf(-(float)rdz, cs, pa.z);
  };
#pragma unroll 1
  for (;;) {
    while (cm == 0u && r < nrec) next_record();
    if (!__any_sync(full, cm != 0u)) break;
    if (cm) {
      const int k1 = 31 - __clz(cm);
      cm ^= 1u << k1;
      const int j1 = cbase + k1;
      const float sy1 = sy, sz1 = sz;
      while (cm == 0u && r < nrec) next_record();
      const bool h2 = cm != 0u;
      const int k2 = h2 ? 31 - __clz(cm) : k1;
      if (h2) cm ^= 1u << k2;
      const int j2 = h2 ? cbase + k2 : j1;
      const float4 pb1 = posc[j1];
      const float4 pb2 = posc[j2];
      const float4 vb1 = velrho[j1];
      const float4 vb2 = velrho[j2];
      const float q1 = press[j1], q2 = press[j2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const float4 pb = u ? pb2 : pb1;
        const float4 vb = u ? vb2 : vb1;
        const int j = u ? j2 : j1;
        const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
        const float ry = (u ? sy : sy1) - pb.y, rz = (u ? sz : sz1) - pb.z;
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        if ((u == 0 || h2) && __float_as_uint(r2) - 1u < r2max_u) {
          const bool bfluid = j < jb;
          const float rr = r2 * rsqrtf(r2);
          const float t = fmaf(-hih, rr, 1.f);
          const float t3 = t * t * t;
          const float vx = va.x - vb.x, vy = va.y - vb.y, vz = va.z - vb.z;
          const float vr = fmaf(vx, rx, fmaf(vy, ry, vz * rz));
          const float ib = __fdividef(1.f, vb.w);
          const float sab = va.w + vb.w;
          const float ie = __fdividef(1.f, (r2 + eta2) * sab);
          mur = fmaxf(mur, fabsf(vr * ie * sab));
          const float pi = fminf(vr, 0.f) * ie;
          const float F = t3 * fmaf(kvisc, pi, fmaf(Qa, ib, (u ? q2 : q1) * ia));
          fx = fmaf(F, rx, fx);
          fy = fmaf(F, ry, fy);
          fz = fmaf(F, rz, fz);
          // Eq 17-18 between fluid particles: d = rho_b - rho_a
          const float d = (ddt_on && bfluid) ? vb.w - va.w : 0.f;
          cont = fmaf(t3 * ib, fmaf(va.w, vr, -kddt * d), cont);
          // b: -F r_ab (its r_ba = -r_ab), t^3/rho_a (rho_b v.r + kddt d)
          const float cb = t3 * ia * fmaf(vb.w, vr, kddt * d);
          atomicAdd(&sum[j], make_float4(-F * rx, -F * ry, -F * rz, cb));
          // each particle's own mu_max (an output only when asked for; the
          // Eq 35 minimum needs only the largest over all pairs)
          if (a.mu_out) atomicMax(&mu_bits[j], __float_as_uint(fabsf(vr * ie * sab)));
          if (bfluid) nff++; else nfb++;
        }
      }
    }
  }
  if (afluid) {
    atomicAdd(&sum[i], make_float4(fx, fy, fz, cont));
    atomicMax(&mu_bits[i], __float_as_uint(mur));
  }
  // directed pairs: an unordered fluid pair is two, a fluid-boundary pair is
  // one of each kind
  reduce_case(i < n ? cidx : -1, has, 2u * nff + 2u * nfb, nfb, nfb, kFloatInfBits, false,
              a.dyn);
}

// dv/dt = g - m cw sum.xyz for fluid particles (0 for boundary ones), drho/dt
// = m cw sum.w, mu_max = h max|mu| (fluid), the Eq 35 candidate time step and
// the non-finite flag, per case; clears the sums for the next evaluation.
// A short, memory-latency-bound kernel: each thread takes kFinishPer
// particles (a block's range of kFinishPer x kFinishThreads), all their
// loads issued first; the per-case minimum is merged per warp, then per
// block, so that one atomic per block of one case reaches the same address
// (all warps of the kernel end together).
constexpr int kFinishThreads = 512;
constexpr int kFinishPer = 4;
__global__ void __launch_bounds__(kFinishThreads)
k_sym_finish(const ListArgs a, float4 *__restrict__ sum, unsigned *__restrict__ mu_bits) {
  __shared__ int s_case[kFinishThreads / 32];
  __shared__ unsigned s_dt[kFinishThreads / 32];
  __shared__ unsigned s_bad[kFinishThreads / 32];
  const unsigned full = 0xffffffffu;
  const int n = a.n;
  const int nbits = a.nbits;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * (kFinishThreads * kFinishPer) + threadIdx.x;
  float4 sm[kFinishPer];
  unsigned mb[kFinishPer];
  uint32_t key[kFinishPer];
  int cid[kFinishPer];
#pragma unroll
  for (int k = 0; k < kFinishPer; k++) {
    const int64_t i = base + (int64_t)k * kFinishThreads;
    sm[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    mb[k] = 0u;
    key[k] = key_out(nbits);
    cid[k] = 0;
    if (i < n) {
      sm[k] = sum[i];
      mb[k] = mu_bits[i];
      key[k] = a.keys[i];
      cid[k] = (int)a.cid[i];
    }
  }
  const int nvalid = *a.nvalid_p;
  // lane 0's running per-case minimum of the warp (case -1: none yet)
  int rc = -1;
  unsigned rdt = kFloatInfBits, rbad = 0u;
#pragma unroll
  for (int k = 0; k < kFinishPer; k++) {
    const int64_t i = base + (int64_t)k * kFinishThreads;
    if (i < n) {  // cleared for the next evaluation
      sum[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      mu_bits[i] = 0u;
    }
    const bool has = i < nvalid && key[k] < key_out(nbits);
    const int cidx = cid[k];
    unsigned dtbits = kFloatInfBits;
    bool bad = false;
    if (has) {
      const CaseConst &C = a.cc[cidx];
      const bool afluid = !key_boundary(key[k], nbits);
      const float mcw = C.m * C.cw;
      float4 out;
      float mumax = C.h * __uint_as_float(mb[k]);
      if (afluid) {
        out.x = fmaf(-mcw, sm[k].x, C.g[0]);
        out.y = fmaf(-mcw, sm[k].y, C.g[1]);
        out.z = fmaf(-mcw, sm[k].z, C.g[2]);
        out.w = mcw * sm[k].w;
        const float f = sqrtf(out.x * out.x + out.y * out.y + out.z * out.z);
        const float dtf = f > 0.f ? sqrtf(C.h / f) : INFINITY;
        const float dtcv = C.h / (C.cs0f + mumax);
        bad = !(isfinite(out.x) && isfinite(out.y) && isfinite(out.z) && isfinite(out.w));
        if (a.want_dt) dtbits = __float_as_uint(fminf(dtf, dtcv));
      } else {
        out = make_float4(0.f, 0.f, 0.f, mcw * sm[k].w);
        mumax = 0.f;
        bad = !isfinite(out.w);
      }
      a.ace[i] = out;
      if (a.mu_out) a.mu_out[i] = mumax;
    }
    const int c0 = __shfl_sync(full, has ? cidx : -1, 0);
    const bool uniform = __all_sync(full, has && cidx == c0);
    const unsigned m = __reduce_min_sync(full, dtbits);
    const unsigned anybad = __any_sync(full, bad);
    if (!uniform) {  // a warp across cases (or the tail): each lane for itself
      if (has && dtbits < kFloatInfBits) atomicMin(&a.dyn[cidx].dtmin_bits, dtbits);
      if (has && bad) atomicOr(&a.dyn[cidx].flags, kFlagNaN);
    } else if (lane == 0) {
      if (rc != c0 && rc >= 0) {  // another case: flush the running one
        if (rdt < kFloatInfBits) atomicMin(&a.dyn[rc].dtmin_bits, rdt);
        if (rbad) atomicOr(&a.dyn[rc].flags, kFlagNaN);
        rdt = kFloatInfBits;
        rbad = 0u;
      }
      rc = c0;
      rdt = min(rdt, m);
      rbad |= anybad;
    }
  }
  if (lane == 0) {
    s_case[w] = rc;
    s_dt[w] = rdt;
    s_bad[w] = rbad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = kFinishThreads / 32;
    int cb = -1;
    bool one = true;
    for (int k = 0; k < nw; k++) {
      if (s_case[k] < 0) continue;
      if (cb < 0) cb = s_case[k];
      else if (s_case[k] != cb) one = false;
    }
    if (one && cb >= 0) {  // the block's uniform warps are of one case
      unsigned m = kFloatInfBits, b = 0u;
      for (int k = 0; k < nw; k++) {
        m = min(m, s_dt[k]);
        b |= s_bad[k];
      }
      if (m < kFloatInfBits && m < *(volatile unsigned *)&a.dyn[cb].dtmin_bits)
        atomicMin(&a.dyn[cb].dtmin_bits, m);
      if (b) atomicOr(&a.dyn[cb].flags, kFlagNaN);
    } else {
      for (int k = 0; k < nw; k++) {
        if (s_case[k] < 0) continue;
        if (s_dt[k] < kFloatInfBits) atomicMin(&a.dyn[s_case[k]].dtmin_bits, s_dt[k]);
        if (s_bad[k]) atomicOr(&a.dyn[s_case[k]].flags, kFlagNaN);
      }
    }
  }
}

// The strain pass of the laminar + SPS model (as k_strain) over the target's
// list records, for the half-step state kept in the order and cells of state n.
__global__ void __launch_bounds__(128)
k_strain_list(int n, const int *__restrict__ nvalid_p, const uint32_t *__restrict__ keys,
              const float4 *__restrict__ posc, const float4 *__restrict__ velrho,
              const uint16_t *__restrict__ cid, int nbits, const CaseConst *__restrict__ cc,
              const uint2 *__restrict__ list, int cap, const uint16_t *__restrict__ count,
              float4 *__restrict__ tau4, float2 *__restrict__ tau2) {
  const unsigned full = 0xffffffffu;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nvalid = *nvalid_p;
  const uint32_t key = i < nvalid ? keys[i] : key_out(nbits);
  const int cidx = i < n ? (int)cid[i] : 0;
  const CaseConst &C = cc[cidx];
  const bool act = key < key_out(nbits) && !key_boundary(key, nbits) && C.visc == 1;
  if (__all_sync(full, !act)) {
    if (i < n) {
      tau4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      tau2[i] = make_float2(0.f, 0.f);
    }
    return;
  }
  const float cs = C.csf, hih = C.half_inv_h;
  const unsigned r2max_u = __float_as_uint(C.r2max) - 1u;
  const float4 pa = act ? posc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 va = act ? velrho[i] : make_float4(0.f, 0.f, 0.f, 1.f);
  const int nrec = act ? (int)count[i] : 0;
  const uint2 *__restrict__ mine = list + (int64_t)i * cap;
  float gxx = 0.f, gyy = 0.f, gzz = 0.f, gxy = 0.f, gxz = 0.f, gyz = 0.f;
  int r = 0;
  unsigned cm = 0u;
  int cbase = 0;
  float sy = 0.f, sz = 0.f;
#pragma unroll 1
  for (;;) {
    if (cm == 0u && r < nrec) {
      const uint2 rec = mine[r++];
      cbase = (int)(rec.x & kListIndexMask);
      cm = rec.y;
      int rdy, rdz;
      list_row_decode(rec.x, rdy, rdz);
      sy = fmaf(-(float)rdy, cs, pa.y);
      sz = fmaf(-(float)rdz, cs, pa.z);
    }
    if (!__any_sync(full, cm != 0u)) break;
    if (cm) {
      const int k = 31 - __clz(cm);
      cm ^= 1u << k;
      const int j = cbase + k;
      const float4 pb = posc[j];
      const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
      const float ry = sy - pb.y, rz = sz - pb.z;
      const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      if (__float_as_uint(r2) - 1u < r2max_u) {
        const float4 vb = velrho[j];
        const float t = fmaf(-hih, r2 * rsqrtf(r2), 1.f);
        const float w = t * t * t * __fdividef(1.f, vb.w);
        const float dvx = vb.x - va.x, dvy = vb.y - va.y, dvz = vb.z - va.z;
        gxx = fmaf(w * dvx, rx, gxx);
        gyy = fmaf(w * dvy, ry, gyy);
        gzz = fmaf(w * dvz, rz, gzz);
        gxy = fmaf(w, fmaf(dvx, ry, dvy * rx), gxy);
        gxz = fmaf(w, fmaf(dvx, rz, dvz * rx), gxz);
        gyz = fmaf(w, fmaf(dvy, rz, dvz * ry), gyz);
      }
    }
  }
  if (i >= n) return;
  if (!act) {
    tau4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    tau2[i] = make_float2(0.f, 0.f);
    return;
  }
  sps_tau_from_gradient(C, gxx, gyy, gzz, gxy, gxz, gyz, tau4[i], tau2[i]);
}

// Half step for the list path: state n+1/2 in the same order and the same
// cells as state n (Eq 33-34 as k_predictor); a particle that leaves the
// domain is frozen at state n and moved out of every list's reach.  The
// displacement since the list's build (from ref, else the half step alone)
// must stay within half the skin (kFlagSkin).
template <bool REF>
__global__ void k_predictor_list(int n, const uint32_t *__restrict__ keys_in, State src,
                                 const float4 *__restrict__ ace,
                                 const CaseConst *__restrict__ cc, CaseDyn *__restrict__ dyn,
                                 int nbits, float4 *__restrict__ posc_out,
                                 float4 *__restrict__ velrho_out, uint32_t *__restrict__ keys_out,
                                 float *__restrict__ press, const float4 *__restrict__ ref) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // every load of the particle first (independent: one memory latency)
  const uint32_t k = keys_in[i];
  const float4 p = src.posc[i];
  const float4 v = src.velrho[i];
  const int cidx = src.cid[i];
  const uint8_t code = src.code[i];
  const float4 a = ace[i];
  const float4 r = REF ? ref[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const CaseConst &C = cc[cidx];
  if (k >= key_out(nbits)) {
    posc_out[i] = p;
    velrho_out[i] = v;
    keys_out[i] = k;
    return;
  }
  const CaseDyn &D = dyn[cidx];
  double disp[3];
  float4 vn;
  predictor_core(C, D, code, v, a, disp, vn);
  const float hs = 0.5f * D.skin;
  float dx = (float)disp[0], dy = (float)disp[1], dz = (float)disp[2];
  if (REF) {
    dx = (float)((double)p.x + disp[0]) - r.x;
    dy = (float)((double)p.y + disp[1]) - r.y;
    dz = (float)((double)p.z + disp[2]) - r.z;
  }
  if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > hs * hs) atomicOr(&dyn[cidx].flags, kFlagSkin);
  float4 ptmp;
  bool left;
  (void)move_particle(k, p, disp, C, code != 0, nbits, ptmp, left);
  if (left) {
    posc_out[i] = make_float4(1e30f, 1e30f, 1e30f, p.w);
    velrho_out[i] = v;
    keys_out[i] = key_out(nbits);
    atomicAdd(&dyn[cidx].n_out, 1);
    return;
  }
  posc_out[i] = make_float4((float)((double)p.x + disp[0]), (float)((double)p.y + disp[1]),
                            (float)((double)p.z + disp[2]), p.w);
  velrho_out[i] = vn;
  keys_out[i] = k;
  press[i] = tait_pressure(C, vn.w) / vn.w;  // P/rho of Eq 28 at n+1/2
}

// Full step for the list path, in the order of state n (sn): writes state n+1
// to x (id, case and code copied) and its keys.
__global__ void k_corrector_list(int n, const uint32_t *__restrict__ keys_n,
                                 const uint32_t *__restrict__ keys_half, State sn,
                                 const float4 *__restrict__ velrho_half,
                                 const float4 *__restrict__ ace, const CaseConst *__restrict__ cc,
                                 CaseDyn *__restrict__ dyn, int nbits, State x,
                                 uint32_t *__restrict__ keys_next) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys_n[i];
  const float4 pn = sn.posc[i];
  const float4 vn = sn.velrho[i];
  const int cidx = sn.cid[i];
  const uint8_t code = sn.code[i];
  x.id[i] = sn.id[i];
  x.cid[i] = (uint16_t)cidx;
  x.code[i] = code;
  if (x.ghost) x.ghost[i] = sn.ghost[i];  // mDBC ghost offsets follow the order
  const CaseConst &C = cc[cidx];
  if (k >= key_out(nbits)) {  // frozen before this step, or released
    x.posc[i] = pn;
    x.velrho[i] = vn;
    keys_next[i] = k;
    return;
  }
  if (keys_half[i] >= key_out(nbits)) {  // left at the half step: frozen at state n
    int cx, cy, cz;
    decode_cell(key_cell(k, nbits) - C.cellbase, C.nx, C.ny, cx, cy, cz);
    x.posc[i] = make_float4((float)(cx * C.cs + pn.x), (float)(cy * C.cs + pn.y),
                            (float)(cz * C.cs + pn.z), 0.f);
    x.velrho[i] = vn;
    keys_next[i] = key_out(nbits);
    return;
  }
  float4 pnew, vnew;
  keys_next[i] = corrector_core(C, dyn[cidx], code, k, pn, vn, velrho_half[i].w, ace[i], nbits,
                                cidx, dyn, pnew, vnew);
  x.posc[i] = pnew;
  x.velrho[i] = vnew;
}

// Full step for the list kept across steps.  State n (y: the order and cells
// of the list's build, offsets relative to those cells) goes to state n+1
// twice: in x with normalised cells and keys (the state the API reads and the
// next build sorts), and in place in y, still in the build's cells, with P/rho
// of Eq 28 in press, for the next step's evaluations over the same list.
// The list stays valid for the next step when every particle satisfies
// |r - r_build| + 1.25 (dt_max / 2) |v| <= (skin - 1e-3 h) / 2 (dt_max the
// Eq 35 bound: the displacement at n+1 and the most the next half step
// adds); otherwise, or when a particle leaves the domain, the corrector
// requests a rebuild.
__global__ void k_corrector_reuse(int n, const uint32_t *__restrict__ keys_n,
                                  const uint32_t *__restrict__ keys_half, State y,
                                  const float4 *__restrict__ velrho_half,
                                  const float4 *__restrict__ ace, const float4 *__restrict__ ref,
                                  const CaseConst *__restrict__ cc, CaseDyn *__restrict__ dyn,
                                  int nbits, State x, uint32_t *__restrict__ keys_next,
                                  float *__restrict__ press, ListCtl *__restrict__ ctl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // every load of the particle first (independent: one memory latency)
  const uint32_t k = keys_n[i];
  const float4 pn = y.posc[i];
  const float4 vn = y.velrho[i];
  const int cidx = y.cid[i];
  const uint8_t code = y.code[i];
  const uint32_t kh = keys_half[i];
  const float rho_half = velrho_half[i].w;
  const float4 a = ace[i];
  const float4 r = ref[i];
  x.id[i] = y.id[i];
  x.cid[i] = (uint16_t)cidx;
  x.code[i] = code;
  if (x.ghost) x.ghost[i] = y.ghost[i];  // mDBC ghost offsets follow the order
  const CaseConst &C = cc[cidx];
  if (k >= key_out(nbits)) {  // frozen before this step, or released
    x.posc[i] = pn;
    x.velrho[i] = vn;
    keys_next[i] = k;
    return;
  }
  if (kh >= key_out(nbits)) {  // left at the half step: frozen at state n
    int cx, cy, cz;
    decode_cell(key_cell(k, nbits) - C.cellbase, C.nx, C.ny, cx, cy, cz);
    x.posc[i] = make_float4((float)(cx * C.cs + pn.x), (float)(cy * C.cs + pn.y),
                            (float)(cz * C.cs + pn.z), 0.f);
    x.velrho[i] = vn;
    keys_next[i] = key_out(nbits);
    dyn[cidx].need = 1u;
    ctl->full = 1u;  // the frozen particle moves to the tail of the order
    ctl->rebuild = 1u;
    return;
  }
  const CaseDyn &D = dyn[cidx];
  float4 pnew, vnew;
  double disp[3];
  const uint32_t kn = corrector_core(C, D, code, k, pn, vn, rho_half, a, nbits,
                                     cidx, dyn, pnew, vnew, disp);
  x.posc[i] = pnew;
  x.velrho[i] = vnew;
  keys_next[i] = kn;
  if (kn >= key_out(nbits)) {  // left at the full step: frozen in x
    dyn[cidx].need = 1u;
    ctl->full = 1u;
    ctl->rebuild = 1u;
    return;
  }
  const float4 pu = make_float4((float)((double)pn.x + disp[0]), (float)((double)pn.y + disp[1]),
                                (float)((double)pn.z + disp[2]), pn.w);
  y.posc[i] = pu;
  y.velrho[i] = vnew;
  press[i] = tait_pressure(C, vnew.w) / vnew.w;
  const float dx = pu.x - r.x, dy = pu.y - r.y, dz = pu.z - r.z;
  const float v = sqrtf(fmaf(vnew.x, vnew.x, fmaf(vnew.y, vnew.y, vnew.z * vnew.z)));
  const float e = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + 0.5f * C.list_k * v;
  if (e > 0.5f * (D.skin - 1e-3f * C.h)) {
    dyn[cidx].need = 1u;
    ctl->rebuild = 1u;
  }
}

// Sets the condition of the graph's IF node that guards a list build: the
// rebuild request of the list kept across steps.
__global__ void k_decide(cudaGraphConditionalHandle h, const ListCtl *__restrict__ ctl) {
  cudaGraphSetConditional(h, ctl->rebuild != 0u ? 1u : 0u);
}

// Brute-force check of a neighbour list (an option for tests, off by
// default): for every target of the evaluated state, the pairs inside 2h over
// all particles of its case (boundary targets: fluid neighbours only, Eq 36)
// are counted with the list walk's own arithmetic (cells of the keys, FP32
// offsets) and compared with the pairs its list records yield.  Adds the
// brute-force pairs to ctl->check_pairs and every mismatching target to
// ctl->check_bad.
__global__ void k_list_check(int n, const int *__restrict__ nvalid_p,
                             const uint32_t *__restrict__ keys, const float4 *__restrict__ posc,
                             const uint16_t *__restrict__ cid, const CaseConst *__restrict__ cc,
                             int nbits, const uint2 *__restrict__ list, int cap,
                             const uint16_t *__restrict__ count, ListCtl *__restrict__ ctl,
                             int half, const uint32_t *__restrict__ row_keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nvalid = *nvalid_p;
  if (i >= nvalid || i >= n) return;
  const uint32_t k = keys[i];
  if (k >= key_out(nbits)) return;
  const bool afluid = !key_boundary(k, nbits);
  const int cidx = cid[i];
  const CaseConst &C = cc[cidx];
  if (!afluid && C.bmode == 1) return;  // mDBC boundary: no pair terms (Eq 38 instead)
  const float cs = C.csf;
  const unsigned r2max_u = __float_as_uint(C.r2max) - 1u;
  const float4 pa = posc[i];
  int cx, cy, cz;
  decode_cell(key_cell(k, nbits) - C.cellbase, C.nx, C.ny, cx, cy, cz);
  unsigned nb = 0u, nl = 0u;
  for (int j = 0; j < nvalid; j++) {
    const uint32_t kj = keys[j];
    if (cid[j] != cidx || kj >= key_out(nbits) || (!afluid && key_boundary(kj, nbits))) continue;
    if (half && j <= i) continue;  // a half list holds the larger indices only
    int jx, jy, jz;
    decode_cell(key_cell(kj, nbits) - C.cellbase, C.nx, C.ny, jx, jy, jz);
    const float4 pb = posc[j];
    const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
    const float ry = fmaf(-(float)(jy - cy), cs, pa.y) - pb.y;
    const float rz = fmaf(-(float)(jz - cz), cs, pa.z) - pb.z;
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    if (__float_as_uint(r2) - 1u < r2max_u) nb++;
  }
  for (int r = 0; r < (int)count[i]; r++) {
    const uint2 rec = list[(int64_t)i * cap + r];
    const int cbase = row_keys ? (int)rec.x : (int)(rec.x & kListIndexMask);
    int rdy, rdz;
    if (row_keys) {  // wide records: the row from the first candidate's cell
      int bx, by, bz, tx, ty, tz;
      decode_cell(key_cell(row_keys[cbase], nbits) - C.cellbase, C.nx, C.ny, bx, by, bz);
      decode_cell(key_cell(row_keys[i], nbits) - C.cellbase, C.nx, C.ny, tx, ty, tz);
      rdy = by - ty;
      rdz = bz - tz;
    } else {
      list_row_decode(rec.x, rdy, rdz);
    }
    const float sy = fmaf(-(float)rdy, cs, pa.y);
    const float sz = fmaf(-(float)rdz, cs, pa.z);
    for (unsigned m = rec.y; m; m &= m - 1u) {
      const float4 pb = posc[cbase + __ffs(m) - 1];
      const float rx = fmaf(pa.w - pb.w, cs, pa.x - pb.x);
      const float ry = sy - pb.y, rz = sz - pb.z;
      const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      if (__float_as_uint(r2) - 1u < r2max_u) nl++;
    }
  }
  atomicAdd(&ctl->check_pairs, (unsigned long long)nb);
  if (nb != nl) atomicAdd(&ctl->check_bad, 1ull);
}

// ---- Verlet scheme ---------------------------------------------------------------

// One Verlet step (Eq 30, or Eq 31 when the case's count of completed steps
// is a multiple of N_S) from the sorted state n (src, with v^{n-1}, rho^{n-1}
// in src.vrprev) and F^n, R^n (ace) to state n+1 in dst, same order:
//   r^{n+1} = r^n + dt v^n + dt^2 F^n / 2            (FP64 displacement)
//   v^{n+1} = v^{n-1} + 2 dt F^n   |  v^n + dt F^n    (Eq 30 | Eq 31)
//   rho^{n+1} = rho^{n-1} + 2 dt R^n | rho^n + dt R^n
// and v^n, rho^n become dst.vrprev.  Boundary particles: density as above
// (clamped >= rho0 when set), fixed ones keep r and v, moving ones follow
// Eq 37 at t + dt.  Cases that take no step (dt = 0) are copied unchanged.
// REUSE (the list kept across steps): src is the state in the list build's
// order and cells; state n+1 also goes into src in place (those cells, P/rho
// to press), and the step requests a rebuild (ctl) when a particle is farther
// than (skin - 1e-3 h) / 2 from its build position (ref) or leaves the domain.
template <bool REUSE>
__global__ void k_verlet(int n, const uint32_t *__restrict__ keys_in, State src,
                         const float4 *__restrict__ ace, const CaseConst *__restrict__ cc,
                         CaseDyn *__restrict__ dyn, int nbits, State dst,
                         uint32_t *__restrict__ keys_out, const float4 *__restrict__ ref = nullptr,
                         float *__restrict__ press = nullptr, ListCtl *__restrict__ ctl = nullptr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys_in[i];
  const float4 p = src.posc[i];
  const float4 v = src.velrho[i];
  const float4 vp = src.vrprev[i];
  const int cidx = src.cid[i];
  const uint8_t code = src.code[i];
  dst.id[i] = src.id[i];
  dst.cid[i] = (uint16_t)cidx;
  dst.code[i] = code;
  if (src.ghost) dst.ghost[i] = src.ghost[i];
  const CaseConst &C = cc[cidx];
  const CaseDyn &D = dyn[cidx];
  const double dt = D.dt;
  if (k >= key_out(nbits) || !(dt > 0.0)) {  // frozen, released or not stepping
    dst.posc[i] = p;
    dst.velrho[i] = v;
    dst.vrprev[i] = vp;
    keys_out[i] = k;
    return;
  }
  const bool eq31 = (D.step % C.verlet_steps) == 0;
  const float dtf = (float)dt;
  const float4 a = ace[i];
  const float4 base = eq31 ? v : vp;  // v, rho at n (Eq 31) or n-1 (Eq 30)
  const float fdt = eq31 ? dtf : 2.f * dtf;
  float rho = fmaf(fdt, a.w, base.w);
  double disp[3];
  float4 vnew;
  if (code == 0) {
    vnew = make_float4(fmaf(fdt, a.x, base.x), fmaf(fdt, a.y, base.y), fmaf(fdt, a.z, base.z), rho);
    const double hdt2 = 0.5 * dt * dt;
    disp[0] = fma(hdt2, (double)a.x, dt * (double)v.x);
    disp[1] = fma(hdt2, (double)a.y, dt * (double)v.y);
    disp[2] = fma(hdt2, (double)a.z, dt * (double)v.z);
  } else {
    if (C.clamp && rho < C.rho0) rho = C.rho0;
    if (code >= 2) {
      const int g = code - 2;
      const double d = D.mot[g][2];
      const float vm = (float)D.mot[g][3];
      disp[0] = d * C.mot_axis[g][0];
      disp[1] = d * C.mot_axis[g][1];
      disp[2] = d * C.mot_axis[g][2];
      vnew = make_float4(vm * C.mot_axis[g][0], vm * C.mot_axis[g][1], vm * C.mot_axis[g][2],
                         rho);
    } else {
      disp[0] = disp[1] = disp[2] = 0.0;
      vnew = make_float4(v.x, v.y, v.z, rho);
    }
  }
  float4 pnew;
  bool left;
  const uint32_t kn = move_particle(k, p, disp, C, code != 0, nbits, pnew, left);
  if (left) atomicAdd(&dyn[cidx].n_out, 1);  // frozen at state n+1
  dst.posc[i] = pnew;
  dst.velrho[i] = vnew;
  dst.vrprev[i] = v;
  keys_out[i] = kn;
  if (REUSE) {
    if (left) {
      dyn[cidx].need = 1u;
      ctl->full = 1u;
      ctl->rebuild = 1u;
      return;
    }
    const float4 pu = make_float4((float)((double)p.x + disp[0]), (float)((double)p.y + disp[1]),
                                  (float)((double)p.z + disp[2]), p.w);
    src.posc[i] = pu;
    src.velrho[i] = vnew;
    src.vrprev[i] = v;
    press[i] = tait_pressure(C, vnew.w) / vnew.w;
    const float4 r = ref[i];
    const float dx = pu.x - r.x, dy = pu.y - r.y, dz = pu.z - r.z;
    if (sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) > 0.5f * (D.skin - 1e-3f * C.h)) {
      dyn[cidx].need = 1u;
      ctl->rebuild = 1u;
    }
  }
}

// ---- read-out ------------------------------------------------------------------

__device__ __forceinline__ void cell_position(uint32_t k, const float4 &p, const CaseConst &C,
                                              int nbits, double &x, double &y, double &z) {
  if (k >= key_out(nbits)) {
    x = (double)p.x;
    y = (double)p.y;
    z = (double)p.z;
  } else {
    int cx, cy, cz;
    decode_cell(key_cell(k, nbits) - C.cellbase, C.nx, C.ny, cx, cy, cz);
    x = cx * C.cs + (double)p.x;
    y = cy * C.cs + (double)p.y;
    z = cz * C.cs + (double)p.z;
  }
}

__global__ void k_export(int n, const uint32_t *__restrict__ keys, State st,
                         const CaseConst *__restrict__ cc, int slot, uint32_t id_base,
                         int nbits, double *__restrict__ pos, float *__restrict__ vel,
                         float *__restrict__ rho, float *__restrict__ press) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || st.cid[i] != slot) return;
  const uint32_t k = keys[i];
  if (k == key_dead(nbits)) return;
  const CaseConst &C = cc[slot];
  const uint32_t lid = st.id[i] - id_base;
  const float4 p = st.posc[i];
  const float4 v = st.velrho[i];
  double x, y, z;
  cell_position(k, p, C, nbits, x, y, z);
  if (pos) {
    pos[3 * lid] = C.origin[0] + x;
    pos[3 * lid + 1] = C.origin[1] + y;
    pos[3 * lid + 2] = C.origin[2] + z;
  }
  if (vel) {
    vel[3 * lid] = v.x;
    vel[3 * lid + 1] = v.y;
    vel[3 * lid + 2] = v.z;
  }
  if (rho) rho[lid] = v.w;
  if (press) press[lid] = tait_pressure(C, v.w);
}

// Raw import (checkpoint restore).
__global__ void k_import_raw(int n, const int32_t *__restrict__ cell,
                             const float4 *__restrict__ posc, const float4 *__restrict__ velrho,
                             const uint8_t *__restrict__ type, const int32_t *__restrict__ group,
                             int slot, uint32_t id_base, const CaseConst *__restrict__ cc,
                             int nbits, State st, uint32_t *__restrict__ keys, int dst0,
                             const float *__restrict__ ghost) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (st.ghost)
    st.ghost[dst0 + i] = ghost ? make_float4(ghost[3 * i], ghost[3 * i + 1], ghost[3 * i + 2], 0.f)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
  const CaseConst &C = cc[slot];
  uint8_t code = type[i] == 0 ? 0 : (group && group[i] >= 0 ? (uint8_t)(2 + group[i]) : 1);
  int d = dst0 + i;
  keys[d] = cell[i] < 0 ? key_out(nbits)
                        : key_make(C.cellbase + (uint32_t)cell[i], code != 0, nbits);
  st.posc[d] = posc[i];
  st.velrho[d] = velrho[i];
  if (st.vrprev) st.vrprev[d] = velrho[i];
  st.id[d] = id_base + (uint32_t)i;
  st.cid[d] = (uint16_t)slot;
  st.code[d] = code;
}

// Scatter per-particle results of the sorted order to the original order.
__global__ void k_scatter_forces(int n, const uint16_t *__restrict__ cid,
                                 const uint32_t *__restrict__ id, int slot, uint32_t id_base,
                                 const int *__restrict__ nvalid_p, const float4 *__restrict__ ace,
                                 const float *__restrict__ mu, float *__restrict__ acc_out,
                                 float *__restrict__ drho_out, float *__restrict__ mu_out,
                                 const uint32_t *__restrict__ keys, int nbits) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cid[i] != slot) return;
  const uint32_t lid = id[i] - id_base;
  // keys (or null): the evaluated state's keys; a particle frozen there has no forces
  const bool valid = i < *nvalid_p && (!keys || keys[i] < key_out(nbits));
  const float4 a = valid ? ace[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  if (acc_out) {
    acc_out[3 * lid] = a.x;
    acc_out[3 * lid + 1] = a.y;
    acc_out[3 * lid + 2] = a.z;
  }
  if (drho_out) drho_out[lid] = a.w;
  if (mu_out) mu_out[lid] = valid ? mu[i] : 0.f;
}

// Neighbour count and id fingerprint over the pairs that the interaction
// evaluates (a in F: b in P; a in B: b in F), with the same FP32 distance
// test, visiting every cell of the (2M+1)^3 block.
__device__ __forceinline__ unsigned long long splitmix64_fin(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__global__ void k_pair_stats(int n, const int *__restrict__ nvalid_p,
                             const uint32_t *__restrict__ keys, State st,
                             const uint32_t *__restrict__ cstart, uint32_t cap1, int nbits,
                             const CaseConst *__restrict__ cc, int slot, uint32_t id_base,
                             long long *__restrict__ count, unsigned long long *__restrict__ hash) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *nvalid_p || st.cid[i] != slot) return;
  const CaseConst &C = cc[slot];
  const uint32_t key = keys[i];
  const bool afluid = !key_boundary(key, nbits);
  const int gc = (int)key_cell(key, nbits), nx = C.nx, nxy = C.nx * C.ny, M = C.margin;
  const float4 pa = st.posc[i];
  long long cnt = 0;
  unsigned long long h = 0;
  for (int dz = -M; dz <= M; dz++)
    for (int dy = -M; dy <= M; dy++) {
      const int c0 = gc + dz * nxy + dy * nx - M, c1 = c0 + 2 * M + 1;
      const float sy = fmaf(-(float)dy, C.csf, pa.y), sz = fmaf(-(float)dz, C.csf, pa.z);
      for (int part = 0; part < (afluid ? 2 : 1); part++) {
        const unsigned j0 = cstart[part * cap1 + c0], j1 = cstart[part * cap1 + c1];
        for (unsigned j = j0; j < j1; j++) {
          const float4 pb = st.posc[j];
          const float rx = fmaf(pa.w - pb.w, C.csf, pa.x - pb.x);
          const float ry = sy - pb.y, rz = sz - pb.z;
          const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
          if (r2 < C.r2max && r2 > 0.f) {
            cnt++;
            h += splitmix64_fin((unsigned long long)(st.id[j] - id_base));
          }
        }
      }
    }
  const uint32_t lid = st.id[i] - id_base;
  count[lid] = cnt;
  hash[lid] = h;
}

// FP64 diagnostics of one case: per-block partials (fixed order), then a
// single block sums the partials in block order: deterministic.
__global__ void k_diag_partial(int n, const uint32_t *__restrict__ keys, State st,
                               const CaseConst *__restrict__ cc, int slot, int nbits,
                               double *__restrict__ part) {
  __shared__ double sh[8][256];
  const CaseConst &C = cc[slot];
  double v[8] = {0, 0, 0, 0, 0, 0, -1e300, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (st.cid[i] != slot) continue;
    const uint32_t k = keys[i];
    if (k == key_dead(nbits)) continue;
    v[0] += 1.0;  // particle count; total mass = count * m (Eq 14)
    if (k >= key_out(nbits)) {
      v[7] += 1.0;
      continue;
    }
    if (st.code[i] != 0) continue;
    const float4 q = st.velrho[i];
    const double m = C.m_d;
    v[1] += 0.5 * m * ((double)q.x * q.x + (double)q.y * q.y + (double)q.z * q.z);
    v[2] += m * q.x;
    v[3] += m * q.y;
    v[4] += m * q.z;
    v[5] += 1.0;
    double x, y, z;
    cell_position(k, st.posc[i], C, nbits, x, y, z);
    x += C.origin[0];
    if (x > v[6]) v[6] = x;
  }
  for (int q = 0; q < 8; q++) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 8; q++) {
        if (q == 6)
          sh[q][threadIdx.x] = fmax(sh[q][threadIdx.x], sh[q][threadIdx.x + s]);
        else
          sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
      }
    __syncthreads();
  }
  if (threadIdx.x < 8) part[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

// The blocks' partial sums combined by 256 threads (32 per quantity), in a
// fixed order, so the result does not depend on timing.
__global__ void __launch_bounds__(256)
k_diag_final(int nparts, const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double sh[256];
  const int q = threadIdx.x & 7, g = threadIdx.x >> 3;  // quantity, group of 32
  double v = q == 6 ? -1e300 : 0.0;
  for (int b = g; b < nparts; b += 32) {
    const double x = part[b * 8 + q];
    v = q == 6 ? fmax(v, x) : v + x;
  }
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int st = 16; st > 0; st >>= 1) {
    if (g < st) {
      const double x = sh[(g + st) * 8 + q];
      sh[g * 8 + q] = q == 6 ? fmax(sh[g * 8 + q], x) : sh[g * 8 + q] + x;
    }
    __syncthreads();
  }
  if (threadIdx.x < 8) out[threadIdx.x] = sh[threadIdx.x];
}

// Release: particles of a slot get the dead key and leave at the next sort.
__global__ void k_release(int n, const uint16_t *__restrict__ cid, int slot, int nbits,
                          uint32_t *__restrict__ keys) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && cid[i] == slot) keys[i] = key_dead(nbits);
}

// ---- launchers ---------------------------------------------------------------

static inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

void launch_upload(int n, const double *pos, const float *vel, const float *rho,
                   const uint8_t *type, const int32_t *group, int slot, uint32_t id_base,
                   const CaseConst *cc, CaseDyn *dyn, int nbits, State st, uint32_t *keys,
                   int dst0, const float *ghost, cudaStream_t s) {
  if (n > 0)
    k_upload<<<nblk(n, 256), 256, 0, s>>>(n, pos, vel, rho, type, group, slot, id_base, cc,
                                          dyn, nbits, st, keys, dst0, ghost);
}

void launch_reorder(int n, const uint32_t *perm, const uint32_t *keys_sorted,
                    const float4 *posc, const float4 *velrho, const uint32_t *id,
                    const uint16_t *cid, const uint8_t *code, const float4 *vrprev,
                    const float4 *ghost, State dst, float *press, const CaseConst *cc,
                    CaseDyn *dyn, int nbits, cudaStream_t s, const float4 *ref_src,
                    float4 *ref_dst) {
  if (n > 0)
    k_reorder<<<nblk(n, 256), 256, 0, s>>>(n, perm, keys_sorted, posc, velrho, id, cid, code,
                                           vrprev, ghost, dst, press, cc, dyn, nbits, ref_src,
                                           ref_dst);
}

size_t cells_temp_words(int64_t cap_cells) {
  return (size_t)((2 * (cap_cells + 1) + kFillBlock - 1) / kFillBlock) + 1;
}

int launch_cells(int n, const uint32_t *keys, uint32_t *cstart, int64_t cap_cells, int nbits,
                 int *nvalid, uint32_t *tmp, cudaStream_t s) {
  const int64_t len = 2 * (cap_cells + 1);
  const int nb = (int)((len + kFillBlock - 1) / kFillBlock);
  cudaMemsetAsync(nvalid, 0, sizeof(int), s);
  if (n > 0) {
    cudaMemsetAsync(cstart, 0xff, sizeof(uint32_t) * (size_t)len, s);
    k_mark<<<nblk(n, 256), 256, 0, s>>>(n, keys, cstart, (uint32_t)(cap_cells + 1), nbits,
                                        nvalid);
  } else {
    cudaMemsetAsync(cstart, 0, sizeof(uint32_t) * (size_t)len, s);
  }
  k_fill_block<<<nb, kFillThreads, 0, s>>>(cstart, len, tmp);
  k_fill_carry<<<1, 1024, 0, s>>>(tmp, nb);
  k_fill_apply<<<nblk(len, 256), 256, 0, s>>>(cstart, len, tmp);
  return n > 0 ? 4 : 3;
}

void launch_interact(int margin, int variant, int n, const int *nvalid, const uint32_t *keys,
                     const float4 *posc, const float4 *velrho, const float *press,
                     const uint16_t *cid, const uint32_t *cstart, int64_t cap_cells, int nbits,
                     const CaseConst *cc, CaseDyn *dyn, float4 *ace, float *mu, int want_dt,
                     bool ext, float4 *tau4, float2 *tau2, cudaStream_t s) {
  if (n <= 0) return;
  const int b = 128;
  const uint32_t cap1 = (uint32_t)(cap_cells + 1);
#define SPH_PI_ARGS                                                                      \
  n, nvalid, keys, posc, velrho, press, cid, cstart, cap1, nbits, cc, dyn, ace, mu, want_dt
  if (ext) {
    // extended physics: strain pass (tau, when a laminar + SPS case is
    // present: tau4 != null), then the compacted pair loop with the Eq 19
    // and Eq 23-27 terms
#define SPH_EXT(MM)                                                                            \
  if (tau4)                                                                                    \
    k_strain<MM><<<nblk(n, b), b, 0, s>>>(n, nvalid, keys, posc, velrho, cid, cstart, cap1,  \
                                          nbits, cc, tau4, tau2);                           \
  if (tau4)                                                                                    \
    k_interact<MM, 0, 2><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS, tau4, tau2);                    \
  else                                                                                         \
    k_interact<MM, 0, 1><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS, tau4, tau2);
    if (margin == 1) {
      SPH_EXT(1)
    } else if (margin == 3) {
      SPH_EXT(3)
    } else {
      SPH_EXT(2)
    }
#undef SPH_EXT
  } else if (margin == 1) {
    if (variant == 6)
      k_interact_tile<1><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
    else if (variant == 2)
      k_interact_q<1><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
    else if (variant == 1)
      k_interact<1, 1><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
    else
      k_interact<1, 0><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
  } else if (margin == 3) {
    if (variant == 6)
      k_interact_tile<3><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
    else if (variant == 2)
      k_interact_q<3><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
    else if (variant == 1)
      k_interact<3, 1><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
    else
      k_interact<3, 0><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
  } else {
    if (variant == 6)
      k_interact_tile<2><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
    else if (variant == 2)
      k_interact_q<2><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
    else if (variant == 1)
      k_interact<2, 1><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
    else
      k_interact<2, 0><<<nblk(n, b), b, 0, s>>>(SPH_PI_ARGS);
  }
#undef SPH_PI_ARGS
}

void launch_dt(int ncases, const CaseConst *cc, CaseDyn *dyn, cudaStream_t s) {
  k_dt<<<nblk(ncases, 64), 64, 0, s>>>(ncases, cc, dyn);
}

void launch_end_step(int ncases, const CaseConst *cc, CaseDyn *dyn, cudaStream_t s) {
  k_end_step<<<nblk(ncases, 64), 64, 0, s>>>(ncases, cc, dyn);
}

void launch_predictor(int n, const uint32_t *keys_in, State src, const float4 *ace,
                      const CaseConst *cc, CaseDyn *dyn, int nbits, float4 *posc_out,
                      float4 *velrho_out, uint32_t *keys_out, cudaStream_t s) {
  if (n > 0)
    k_predictor<<<nblk(n, 256), 256, 0, s>>>(n, keys_in, src, ace, cc, dyn, nbits, posc_out,
                                             velrho_out, keys_out);
}

void launch_corrector(int n, const uint32_t *perm2, const uint32_t *keys_half,
                      const uint32_t *keys_n, State sn, State x, const float4 *ace,
                      const CaseConst *cc, CaseDyn *dyn, int nbits, uint32_t *keys_next,
                      cudaStream_t s) {
  if (n > 0)
    k_corrector<<<nblk(n, 256), 256, 0, s>>>(n, perm2, keys_half, keys_n, sn, x, ace, cc, dyn,
                                             nbits, keys_next);
}

void launch_mdbc(int margin, int n, const int *nvalid, const uint32_t *keys, State st,
                 float *press, const uint32_t *cstart, int nbits, const CaseConst *cc,
                 const CaseDyn *dyn, int stage, cudaStream_t s, bool list) {
  if (n <= 0) return;
#define SPH_MD(MM, LL)                                                                    \
  k_mdbc<MM, LL><<<nblk(n, 128), 128, 0, s>>>(n, nvalid, keys, st, press, cstart, nbits, cc, \
                                              dyn, stage)
  if (margin == 1) {
    if (list) SPH_MD(1, true); else SPH_MD(1, false);
  } else if (margin == 3) {
    if (list) SPH_MD(3, true); else SPH_MD(3, false);
  } else {
    if (list) SPH_MD(2, true); else SPH_MD(2, false);
  }
#undef SPH_MD
}

void launch_interact_list(int n, const int *nvalid, const uint32_t *keys, const float4 *posc,
                          const float4 *velrho, const float *press, const uint16_t *cid,
                          const uint32_t *cstart, int64_t cap_cells, int nbits,
                          const CaseConst *cc, CaseDyn *dyn, float4 *ace, int want_dt,
                          const uint2 *list, int cap, const uint16_t *count, bool ext,
                          float4 *tau4, float2 *tau2, cudaStream_t s, float *mu, int block,
                          int lanes, float4 *sym_sum, unsigned *sym_mu,
                          const uint32_t *wide_keys) {
  if (n <= 0) return;
  if (lanes != 2 && lanes != 4 && lanes != 8) lanes = 1;
  const ListArgs a{n,     nvalid, keys,  posc,  velrho, press,  cid,  cstart,
                   (uint32_t)(cap_cells + 1), nbits, cc, dyn,  ace,  want_dt, list,
                   cap,   count,  tau4,  tau2,  mu,     wide_keys};
  if (wide_keys) {  // wide records: the default physics only, one thread per target
    if (sym_sum) {
      k_interact_sym<1><<<nblk(n, 128), 128, 0, s>>>(a, sym_sum, sym_mu);
      k_sym_finish<<<nblk(n, kFinishThreads * kFinishPer), kFinishThreads, 0, s>>>(
          a, sym_sum, sym_mu);
    } else {
      k_interact_list<0, 1, 1><<<nblk(n, 128), 128, 0, s>>>(a);
    }
    return;
  }
  if (sym_sum && !ext && !tau4) {  // each pair once, then the per-particle values
    k_interact_sym<0><<<nblk(n, 128), 128, 0, s>>>(a, sym_sum, sym_mu);
    k_sym_finish<<<nblk(n, kFinishThreads * kFinishPer), kFinishThreads, 0, s>>>(a, sym_sum,
                                                                                 sym_mu);
    return;
  }
  if (tau4)  // laminar + SPS cases present: strain pass over the list first
    k_strain_list<<<nblk(n, 128), 128, 0, s>>>(n, nvalid, keys, posc, velrho, cid, nbits, cc,
                                               list, cap, count, tau4, tau2);
  // G = lanes threads per target; block size 128 (default) to 1024 for the
  // default kernel (EXT 1 and 2: 128, by their registers)
  const int b0 = block >= 128 && block <= 1024 && block % 32 == 0 ? block : 128;
  const int64_t nt = (int64_t)n * lanes;
  const int g1 = (int)((nt + 127) / 128), g0 = (int)((nt + b0 - 1) / b0);
#define SPH_LIST(EXT, GRID, BLK)                                                      \
  switch (lanes) {                                                                  \
    case 2: k_interact_list<EXT, 2><<<GRID, BLK, 0, s>>>(a); break;                 \
    case 4: k_interact_list<EXT, 4><<<GRID, BLK, 0, s>>>(a); break;                 \
    case 8: k_interact_list<EXT, 8><<<GRID, BLK, 0, s>>>(a); break;                 \
    default: k_interact_list<EXT, 1><<<GRID, BLK, 0, s>>>(a); break;                \
  }
  if (tau4) {
    SPH_LIST(2, g1, 128)
  } else if (ext) {
    SPH_LIST(1, g1, 128)
  } else {
    SPH_LIST(0, g0, b0)
  }
#undef SPH_LIST
}

void launch_list_begin(int ncases, const CaseConst *cc, CaseDyn *dyn, ListCtl *ctl,
                       float extra, int fresh_all, const uint32_t *cstart, int64_t cap_cells,
                       cudaStream_t s) {
  k_list_begin<<<(ncases + 127) / 128, 128, 0, s>>>(ncases, cc, dyn, ctl, extra, fresh_all,
                                                     cstart, (uint32_t)(cap_cells + 1));
}

void launch_select(int n, const uint16_t *cid, const CaseConst *cc, const CaseDyn *dyn,
                   const uint32_t *keys_build, const float4 *posc_build, uint32_t *keys,
                   float4 *posc, const ListCtl *ctl, cudaStream_t s) {
  if (n > 0)
    k_select<<<nblk(n, 256), 256, 0, s>>>(n, cid, cc, dyn, keys_build, posc_build, keys, posc,
                                          ctl);
}

size_t rb_temp_words(int64_t n) { return (size_t)((n + kRbTile - 1) / kRbTile) + 2; }

void launch_rebuild_sort(int n, const ListCtl *ctl, const uint32_t *keys, State src, State dst,
                         uint32_t *keys_dst, float *press, const CaseConst *cc, CaseDyn *dyn,
                         int nbits, const float4 *ref_src, float4 *ref_dst, uint32_t *tmp,
                         uint32_t *idx, uint32_t *kc, uint32_t *kc_sorted, uint32_t *perm,
                         void *sort_tmp, cudaStream_t s) {
  if (n <= 0) return;
  const int ntiles = (n + kRbTile - 1) / kRbTile;
  int *m = (int *)(tmp + ntiles);
  k_rb_count<<<ntiles, kRbTile, 0, s>>>(n, src.cid, dyn, ctl, tmp);
  k_rb_scan<<<1, 1024, 0, s>>>(ntiles, tmp, m);
  k_rb_compact<<<ntiles, kRbTile, 0, s>>>(n, src.cid, dyn, ctl, tmp, keys, idx, kc);
  radix_sort(kc, kc_sorted, perm, n, nbits, sort_tmp, s, m);
  k_rb_scatter<<<nblk(n, 256), 256, 0, s>>>(n, m, idx, perm, kc_sorted, src, dst, keys_dst,
                                             press, cc, dyn, nbits, ref_src, ref_dst);
}

void launch_need_all(int ncases, CaseDyn *dyn, cudaStream_t s) {
  k_need_all<<<(ncases + 127) / 128, 128, 0, s>>>(ncases, dyn);
}

void launch_build_list(int margin, int n, const int *nvalid, const uint32_t *keys,
                       const float4 *posc, const float4 *velrho, const float *press,
                       const uint16_t *cid, const uint32_t *cstart, int64_t cap_cells, int nbits,
                       const CaseConst *cc, CaseDyn *dyn, float4 *ace, uint2 *list, int cap,
                       uint16_t *count, float4 *ref, const float4 *ref_src, cudaStream_t s,
                       bool half, bool wide) {
  if (n <= 0) return;
  const uint32_t cap1 = (uint32_t)(cap_cells + 1);
#define SPH_BL_ARGS                                                                        \
  n, nvalid, keys, posc, velrho, press, cid, cstart, cap1, nbits, cc, dyn, ace, nullptr, 0, \
      nullptr, nullptr, list, cap, count, ref, ref_src
#define SPH_BL(L)                                                                \
  if (margin == 1)                                                               \
    k_interact<1, 0, 0, L><<<nblk(n, 128), 128, 0, s>>>(SPH_BL_ARGS);           \
  else if (margin == 3)                                                          \
    k_interact<3, 0, 0, L><<<nblk(n, 128), 128, 0, s>>>(SPH_BL_ARGS);           \
  else                                                                           \
    k_interact<2, 0, 0, L><<<nblk(n, 128), 128, 0, s>>>(SPH_BL_ARGS);
  if (wide && half) {
    SPH_BL(7)
  } else if (wide) {
    SPH_BL(6)
  } else if (half) {
    SPH_BL(3)
  } else if (margin == 1)
    k_interact<1, 0, 0, 2><<<nblk(n, 128), 128, 0, s>>>(SPH_BL_ARGS);
  else if (margin == 3)
    k_interact<3, 0, 0, 2><<<nblk(n, 128), 128, 0, s>>>(SPH_BL_ARGS);
  else
    k_interact<2, 0, 0, 2><<<nblk(n, 128), 128, 0, s>>>(SPH_BL_ARGS);
#undef SPH_BL
#undef SPH_BL_ARGS
}

void launch_interact_build(int margin, int n, const int *nvalid, const uint32_t *keys,
                           const float4 *posc, const float4 *velrho, const float *press,
                           const uint16_t *cid, const uint32_t *cstart, int64_t cap_cells,
                           int nbits, const CaseConst *cc, CaseDyn *dyn, float4 *ace,
                           uint2 *list, int cap, uint16_t *count, bool ext, float4 *tau4,
                           float2 *tau2, cudaStream_t s, float *mu) {
  if (n <= 0) return;
  const uint32_t cap1 = (uint32_t)(cap_cells + 1);
#define SPH_IB_ARGS                                                                        \
  n, nvalid, keys, posc, velrho, press, cid, cstart, cap1, nbits, cc, dyn, ace, mu, 1, \
      tau4, tau2, list, cap, count
  if (tau4) {  // laminar + SPS cases: strain pass on state n, then EXT 2
    if (margin == 1) {
      k_strain<1><<<nblk(n, 128), 128, 0, s>>>(n, nvalid, keys, posc, velrho, cid, cstart, cap1,
                                               nbits, cc, tau4, tau2);
      k_interact<1, 0, 2, 1><<<nblk(n, 128), 128, 0, s>>>(SPH_IB_ARGS);
    } else if (margin == 3) {
      k_strain<3><<<nblk(n, 128), 128, 0, s>>>(n, nvalid, keys, posc, velrho, cid, cstart, cap1,
                                               nbits, cc, tau4, tau2);
      k_interact<3, 0, 2, 1><<<nblk(n, 128), 128, 0, s>>>(SPH_IB_ARGS);
    } else {
      k_strain<2><<<nblk(n, 128), 128, 0, s>>>(n, nvalid, keys, posc, velrho, cid, cstart, cap1,
                                               nbits, cc, tau4, tau2);
      k_interact<2, 0, 2, 1><<<nblk(n, 128), 128, 0, s>>>(SPH_IB_ARGS);
    }
  } else if (ext) {
    if (margin == 1)
      k_interact<1, 0, 1, 1><<<nblk(n, 128), 128, 0, s>>>(SPH_IB_ARGS);
    else if (margin == 3)
      k_interact<3, 0, 1, 1><<<nblk(n, 128), 128, 0, s>>>(SPH_IB_ARGS);
    else
      k_interact<2, 0, 1, 1><<<nblk(n, 128), 128, 0, s>>>(SPH_IB_ARGS);
  } else if (margin == 1) {
    k_interact<1, 0, 0, 1><<<nblk(n, 128), 128, 0, s>>>(SPH_IB_ARGS);
  } else if (margin == 3) {
    k_interact<3, 0, 0, 1><<<nblk(n, 128), 128, 0, s>>>(SPH_IB_ARGS);
  } else {
    k_interact<2, 0, 0, 1><<<nblk(n, 128), 128, 0, s>>>(SPH_IB_ARGS);
  }
#undef SPH_IB_ARGS
}

void launch_predictor_list(int n, const uint32_t *keys_in, State src, const float4 *ace,
                           const CaseConst *cc, CaseDyn *dyn, int nbits, float4 *posc_out,
                           float4 *velrho_out, uint32_t *keys_out, float *press,
                           const float4 *ref, cudaStream_t s) {
  if (n <= 0) return;
  if (ref)
    k_predictor_list<true><<<nblk(n, 256), 256, 0, s>>>(n, keys_in, src, ace, cc, dyn, nbits,
                                                        posc_out, velrho_out, keys_out, press, ref);
  else
    k_predictor_list<false><<<nblk(n, 256), 256, 0, s>>>(n, keys_in, src, ace, cc, dyn, nbits,
                                                         posc_out, velrho_out, keys_out, press,
                                                         ref);
}

void launch_corrector_reuse(int n, const uint32_t *keys_n, const uint32_t *keys_half, State y,
                            const float4 *velrho_half, const float4 *ace, const float4 *ref,
                            const CaseConst *cc, CaseDyn *dyn, int nbits, State x,
                            uint32_t *keys_next, float *press, ListCtl *ctl, cudaStream_t s) {
  if (n > 0)
    k_corrector_reuse<<<nblk(n, 256), 256, 0, s>>>(n, keys_n, keys_half, y, velrho_half, ace,
                                                   ref, cc, dyn, nbits, x, keys_next, press,
                                                   ctl);
}

void launch_decide(cudaGraphConditionalHandle h, const ListCtl *ctl, cudaStream_t s) {
  k_decide<<<1, 1, 0, s>>>(h, ctl);
}

void launch_list_check(int n, const int *nvalid, const uint32_t *keys, const float4 *posc,
                       const uint16_t *cid, const CaseConst *cc, int nbits, const uint2 *list,
                       int cap, const uint16_t *count, ListCtl *ctl, cudaStream_t s, bool half,
                       const uint32_t *wide_keys) {
  if (n > 0)
    k_list_check<<<nblk(n, 128), 128, 0, s>>>(n, nvalid, keys, posc, cid, cc, nbits, list, cap,
                                              count, ctl, half ? 1 : 0, wide_keys);
}

void launch_corrector_list(int n, const uint32_t *keys_n, const uint32_t *keys_half, State sn,
                           const float4 *velrho_half, const float4 *ace, const CaseConst *cc,
                           CaseDyn *dyn, int nbits, State x, uint32_t *keys_next,
                           cudaStream_t s) {
  if (n > 0)
    k_corrector_list<<<nblk(n, 256), 256, 0, s>>>(n, keys_n, keys_half, sn, velrho_half, ace, cc,
                                                  dyn, nbits, x, keys_next);
}

void launch_verlet(int n, const uint32_t *keys_in, State src, const float4 *ace,
                   const CaseConst *cc, CaseDyn *dyn, int nbits, State dst, uint32_t *keys_out,
                   cudaStream_t s) {
  if (n > 0)
    k_verlet<false><<<nblk(n, 256), 256, 0, s>>>(n, keys_in, src, ace, cc, dyn, nbits, dst,
                                                 keys_out);
}

void launch_verlet_reuse(int n, const uint32_t *keys_in, State y, const float4 *ace,
                         const CaseConst *cc, CaseDyn *dyn, int nbits, State x,
                         uint32_t *keys_out, const float4 *ref, float *press, ListCtl *ctl,
                         cudaStream_t s) {
  if (n > 0)
    k_verlet<true><<<nblk(n, 256), 256, 0, s>>>(n, keys_in, y, ace, cc, dyn, nbits, x, keys_out,
                                                ref, press, ctl);
}

void launch_export(int n, const uint32_t *keys, State st, const CaseConst *cc, int slot,
                   uint32_t id_base, int nbits, double *pos, float *vel, float *rho,
                   float *press, cudaStream_t s) {
  if (n > 0)
    k_export<<<nblk(n, 256), 256, 0, s>>>(n, keys, st, cc, slot, id_base, nbits, pos, vel, rho,
                                          press);
}

void launch_import_raw(int n, const int32_t *cell, const float4 *posc, const float4 *velrho,
                       const uint8_t *type, const int32_t *group, int slot, uint32_t id_base,
                       const CaseConst *cc, int nbits, State st, uint32_t *keys, int dst0,
                       const float *ghost, cudaStream_t s) {
  if (n > 0)
    k_import_raw<<<nblk(n, 256), 256, 0, s>>>(n, cell, posc, velrho, type, group, slot, id_base,
                                              cc, nbits, st, keys, dst0, ghost);
}

void launch_scatter_forces(int n, const uint16_t *cid, const uint32_t *id, int slot,
                           uint32_t id_base, const int *nvalid, const float4 *ace,
                           const float *mu, float *acc_out, float *drho_out, float *mu_out,
                           cudaStream_t s, const uint32_t *keys, int nbits) {
  if (n > 0)
    k_scatter_forces<<<nblk(n, 256), 256, 0, s>>>(n, cid, id, slot, id_base, nvalid, ace, mu,
                                                  acc_out, drho_out, mu_out, keys, nbits);
}

// tau/rho (sorted order, tau4/tau2) to the original order of one case: [6 n].
__global__ void k_scatter_tau(int n, const uint16_t *__restrict__ cid,
                              const uint32_t *__restrict__ id, int slot,
                              const int *__restrict__ nvalid_p, const float4 *__restrict__ tau4,
                              const float2 *__restrict__ tau2, float *__restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cid[i] != slot) return;
  const bool valid = i < *nvalid_p;
  const float4 a = valid ? tau4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float2 b = valid ? tau2[i] : make_float2(0.f, 0.f);
  float *o = out + 6 * (size_t)id[i];
  o[0] = a.x;
  o[1] = a.y;
  o[2] = a.z;
  o[3] = a.w;
  o[4] = b.x;
  o[5] = b.y;
}

void launch_strain(int margin, int n, const int *nvalid, const uint32_t *keys,
                   const float4 *posc, const float4 *velrho, const uint16_t *cid,
                   const uint32_t *cstart, int64_t cap_cells, int nbits, const CaseConst *cc,
                   float4 *tau4, float2 *tau2, cudaStream_t s) {
  if (n <= 0) return;
  const uint32_t cap1 = (uint32_t)(cap_cells + 1);
  if (margin == 1)
    k_strain<1><<<nblk(n, 128), 128, 0, s>>>(n, nvalid, keys, posc, velrho, cid, cstart, cap1,
                                             nbits, cc, tau4, tau2);
  else if (margin == 3)
    k_strain<3><<<nblk(n, 128), 128, 0, s>>>(n, nvalid, keys, posc, velrho, cid, cstart, cap1,
                                             nbits, cc, tau4, tau2);
  else
    k_strain<2><<<nblk(n, 128), 128, 0, s>>>(n, nvalid, keys, posc, velrho, cid, cstart, cap1,
                                             nbits, cc, tau4, tau2);
}

void launch_scatter_tau(int n, const uint16_t *cid, const uint32_t *id, int slot,
                        const int *nvalid, const float4 *tau4, const float2 *tau2, float *out,
                        cudaStream_t s) {
  if (n > 0)
    k_scatter_tau<<<nblk(n, 256), 256, 0, s>>>(n, cid, id, slot, nvalid, tau4, tau2, out);
}

void launch_pair_stats(int n, const int *nvalid, const uint32_t *keys, State st,
                       const uint32_t *cstart, int64_t cap_cells, int nbits, const CaseConst *cc,
                       int slot, uint32_t id_base, long long *count, unsigned long long *hash,
                       cudaStream_t s) {
  if (n > 0)
    k_pair_stats<<<nblk(n, 128), 128, 0, s>>>(n, nvalid, keys, st, cstart,
                                              (uint32_t)(cap_cells + 1), nbits, cc, slot,
                                              id_base, count, hash);
}

void launch_diag(int n, const uint32_t *keys, State st, const CaseConst *cc, int slot,
                 int nbits, double *part, int nparts, double *out, cudaStream_t s) {
  k_diag_partial<<<nparts, 256, 0, s>>>(n, keys, st, cc, slot, nbits, part);
  k_diag_final<<<1, 256, 0, s>>>(nparts, part, out);
}

void launch_release(int n, const uint16_t *cid, int slot, int nbits, uint32_t *keys,
                    cudaStream_t s) {
  if (n > 0) k_release<<<nblk(n, 256), 256, 0, s>>>(n, cid, slot, nbits, keys);
}

}  // namespace sph
