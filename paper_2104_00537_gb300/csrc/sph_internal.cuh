// sph_internal.cuh -- device-side data layout shared by the CUDA sources of
// libsph.so (not part of the public ABI).
//
// Particle state lives in structure-of-arrays form, sorted by cell key:
//   posc   float4  {offset x, y, z inside the cell, cell x index (as float)}
//   velrho float4  {v x, y, z, rho}
//   press  float   pressure P of Eq 28 (written by the reorder)
//   id     uint32  particle index within its case (caller's order)
//   cid    uint16  case slot of the particle
//   code   uint8   0 fluid, 1 fixed boundary, 2 + g moving boundary group g
// The key of an in-domain particle is (is_boundary << (nbits-1)) | global cell,
// global cell = cellbase of its case + (cz * ny + cy) * nx + cx, so a stable
// sort by key puts all fluid particles first, in cell order, then all boundary
// particles in cell order (Sect. 5.1: particles sorted by the cell they belong
// to); out-of-domain particles carry key_out(nbits), released ones key_dead.
// cstart[t * (cells + 1) + c] is the first sorted index of type t with cell
// >= c, so every run of consecutive cells of one type is one index range.
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

namespace sph {

constexpr int kMaxMotions = 8;

// Constants of one case, read by every kernel (FP64 for the grid and the
// system update, FP32 for the interaction).
struct CaseConst {
  double origin[3];   // grid origin = domain_min - margin * cs
  double cs, inv_cs;  // cell size
  double h_d, cs0_d, cfl, dt_fixed, dt_min, t_end;
  double m_d;  // particle mass rho0 dp^3 (FP64, for the reductions)
  double mot_amp[kMaxMotions], mot_omega[kMaxMotions], mot_phase[kMaxMotions];
  float mot_axis[kMaxMotions][3];
  int32_t nx, ny, nz, margin;
  uint32_t cellbase;  // first global cell of this case
  int32_t nmot, ddt, clamp, visc;  // visc: 0 artificial (Eq 21), 1 laminar + SPS (Eq 23-27)
  int32_t bmode, mdbc_slip;        // bmode: 0 DBC (Eq 36), 1 mDBC (Eq 38-39)
  int32_t max_out, active, n_fluid, verlet_steps;  // verlet_steps: N_S of Eq 31
  float h, csf, r2max, eta2;
  float m, rho0, inv_rho0, btait, gamma;
  float cw;     // -5 a_D / h^2: grad_a W_ab = cw (1 - q/2)^3 r_ab
  float half_inv_h;  // 0.5 / h
  float kvisc;  // -2 alpha cs0 h: rho_a Pi_ab = kvisc rho_a min(v.r,0) / ((r^2+eta^2)(rho_a+rho_b))
  float kddt;   // 2 delta h cs0
  float g[3];
  float cs0f;
  float inv_csf;  // 1 / cs
  float inv_gamma;
  float khyd[3];  // -(rho0 / B) g: P^H_ab / B of Eq 20 is khyd . r_ab
  float hyd_c[3]; // (k-1)/2, (k-2)/3, (k-3)/4 with k = 1/gamma (binomial series)
  float nu0;      // Eq 23
  float sps_cs2;  // (C_S Delta)^2 of Eq 25
  float sps_cl2;  // C_l Delta^2 of Eq 25
  float wk;       // a_D of Eq 11: W = a_D t^4 (5 - 4t), t = 1 - r/(2h)
  float list_k;   // 1.25 x the Eq 35 bound on dt (or the fixed dt): skin = list_k |v|max + 1e-3 h
};

// Mutable per-case values, updated on the device during a step.
struct CaseDyn {
  double t, dt;
  long long step;
  unsigned long long pairs;     // all evaluated ordered pairs
  unsigned long long pairs_fb;  // pairs with a in F and b in B
  unsigned long long pairs_bf;  // pairs with a in B (b in F)
  unsigned int dtmin_bits;  // float bits of min_a min(dt_f, dt_cv) (positive floats order as ints)
  unsigned int flags;       // kFlag*
  int n_out;
  unsigned int v2max_bits;  // float bits of max |v|^2 over in-domain particles at the last reorder
  float skin;               // neighbour-list path: skin of the list built last (set by k_list_begin)
  // list kept across steps, per case: need = the case's list must be rebuilt
  // (set by the corrector, at admission, by the host); lmode = what the
  // current build does for the case (0 keep the records, 1 build from the
  // state, 2 rebuild from the build positions after an index shift);
  // startF / startB = first fluid / boundary index of the case at its build
  unsigned int need, lmode, startF, startB;
  double mot[kMaxMotions][4];  // displacement and velocity at t+dt/2 and t+dt
};

constexpr unsigned kFlagNaN = 1u, kFlagDtMin = 2u, kFlagQuota = 4u;
// neighbour-list path: a target had more records than its list segment
// holds; a displacement since the list's build exceeded half its skin (or
// one step's need exceeded the largest skin the rows cover)
constexpr unsigned kFlagListFull = 8u, kFlagSkin = 16u;
// list record: first candidate index (25 bits) | row code << 25, with the
// row code (dz + 4) * 9 + (dy + 4) for row offsets dy, dz in [-4, 4]
constexpr int kListMaxParticles = 1 << 25;
constexpr uint32_t kListIndexMask = (1u << 25) - 1u;
__host__ __device__ inline uint32_t list_row_code(int dy, int dz) {
  return (uint32_t)((dz + 4) * 9 + (dy + 4)) << 25;
}
__host__ __device__ inline void list_row_decode(uint32_t x, int &dy, int &dz) {
  const int r = (int)(x >> 25);
  const int q = r / 9;
  dz = q - 4;
  dy = r - 9 * q - 4;
}

// Engine-wide control of the neighbour list kept across steps: rebuild is
// requested by the corrector (a case needs a new list) or by the host (cases
// admitted or released, the sorted state overwritten) and cleared by the
// build; full says that the rebuild must re-sort all cases (else only the
// particles of the cases that need a list, within their own index ranges);
// builds counts the rebuild events; check_pairs / check_bad are the
// optional brute-force check of the list.
struct ListCtl {
  unsigned int rebuild;
  unsigned int full;  // the rebuild must re-sort every case: index ranges may move
                      // (a particle left the domain, cases were admitted or
                      // released, or the sorted state was overwritten)
  unsigned long long builds;
  unsigned long long check_pairs;  // pairs inside 2h found by brute force
  unsigned long long check_bad;    // targets whose brute-force count differs from the list's
};
// Readable entries of posc/velrho/press past the last particle, so that a
// warp may test 32 candidates at a time without per-candidate bounds checks.
constexpr int64_t kReadPad = 1024;
constexpr uint32_t kFloatInfBits = 0x7f800000u;

__host__ __device__ inline uint32_t key_out(int nbits) { return (1u << nbits) - 2u; }
__host__ __device__ inline uint32_t key_dead(int nbits) { return (1u << nbits) - 1u; }
__host__ __device__ inline uint32_t key_bbit(int nbits) { return 1u << (nbits - 1); }
__host__ __device__ inline uint32_t key_make(uint32_t gcell, bool boundary, int nbits) {
  return gcell | (boundary ? key_bbit(nbits) : 0u);
}
__host__ __device__ inline uint32_t key_cell(uint32_t k, int nbits) { return k & (key_bbit(nbits) - 1u); }
__host__ __device__ inline bool key_boundary(uint32_t k, int nbits) { return (k & key_bbit(nbits)) != 0u; }
// smallest nbits with 2^(nbits-1) >= cells + 2, so that key_out exceeds every boundary key
__host__ __device__ inline int key_bits(int64_t cells) {
  int b = 2;
  while ((int64_t(1) << (b - 1)) < cells + 2) b++;
  return b;
}

// Device arrays of one state buffer.
struct State {
  float4 *posc;
  float4 *velrho;
  uint32_t *id;
  uint16_t *cid;
  uint8_t *code;
  float4 *vrprev;  // Verlet scheme only (else null): v^{n-1}, rho^{n-1} of Eq 30
  float4 *ghost;   // mDBC only (else null): ghost offset r_G - r_B (xyz) of Eq 38
};

// Sets the message returned by sph_last_error() (defined in sph_api.cu).
void set_last_error(const std::string &msg);

// ---- launchers (defined in the .cu files) --------------------------------
// Radix sort geometry: keys per tile (block) and digit values per 8-bit pass.
constexpr int64_t kSortTile = 2048;
constexpr int64_t kSortRadix = 256;
// Scratch bytes of radix_sort for n keys: key and index ping-pong buffers,
// per-tile digit histograms and digit totals, each rounded up to 256 bytes.
constexpr size_t sort_temp_bytes(int64_t n) {
  return (size_t)(((n * 4 + 255) / 256) * 256) * 2 +
         (size_t)(((((n + kSortTile - 1) / kSortTile) > 0 ? (n + kSortTile - 1) / kSortTile : 1) *
                       kSortRadix * 4 + 255) / 256 * 256) +
         (size_t)(kSortRadix * 4);
}
size_t radix_sort_temp_bytes(int64_t n);
// Stable LSD sort of keys_in[0,n) by their low 8 ceil(nbits/8) bits (one
// pass per 8-bit digit; keys below 2^nbits sort by value); writes the sorted
// keys and the permutation (source index of each output).  keys_in, keys_out,
// perm_out and temp must not overlap.
// n_dev (or null): the number of keys, at most n, read on the device when
// the kernels run (grids and scratch are sized for n).
void radix_sort(const uint32_t *keys_in, uint32_t *keys_out, uint32_t *perm_out,
                int n, int nbits, void *temp, cudaStream_t s, const int *n_dev = nullptr);

}  // namespace sph
