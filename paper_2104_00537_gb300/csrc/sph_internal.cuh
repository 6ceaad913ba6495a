// sph_internal.cuh -- device-side data layout shared by the CUDA sources of
// libsph.so (not part of the public ABI).
//
// Particle state lives in structure-of-arrays form, sorted by cell key:
//   posc   float4  {offset x, y, z inside the cell, pressure P (Eq 28)}
//   velrho float4  {v x, y, z, rho}
//   id     uint32  particle index in upload order
//   cid    uint16  case slot of the particle
//   code   uint8   0 fluid, 1 fixed boundary, 2 + g moving boundary group g
// The key of a particle is 2 * (cellbase of its case + linear cell) + is_boundary,
// with linear cell = (cz * ny + cy) * nx + cx; out-of-domain particles carry
// key_out(nbits) and released particles key_dead(nbits), so a stable sort by
// key yields the neighbour-list order of Sect. 5.1 for all cases at once.
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
  int32_t nmot, ddt, clamp;
  int32_t max_out, active, n_fluid, pad_;
  float h, csf, r2max, eta2;
  float m, rho0, inv_rho0, btait, gamma;
  float cw;     // -5 a_D / h^2: grad_a W_ab = cw (1 - q/2)^3 r_ab
  float half_inv_h;  // 0.5 / h
  float kvisc;  // -2 alpha cs0 h: rho_a Pi_ab = kvisc rho_a min(v.r,0) / ((r^2+eta^2)(rho_a+rho_b))
  float kddt;   // 2 delta h cs0
  float g[3];
  float cs0f;
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
  int pad_;
  double mot[kMaxMotions][4];  // displacement and velocity at t+dt/2 and t+dt
};

constexpr unsigned kFlagNaN = 1u, kFlagDtMin = 2u, kFlagQuota = 4u;
constexpr uint32_t kFloatInfBits = 0x7f800000u;

__host__ __device__ inline uint32_t key_out(int nbits) { return (1u << nbits) - 2u; }
__host__ __device__ inline uint32_t key_dead(int nbits) { return (1u << nbits) - 1u; }

// Device arrays of one state buffer.
struct State {
  float4 *posc;
  float4 *velrho;
  uint32_t *id;
  uint16_t *cid;
  uint8_t *code;
};

// Sets the message returned by sph_last_error() (defined in sph_api.cu).
void set_last_error(const std::string &msg);

// ---- launchers (defined in the .cu files) --------------------------------
size_t radix_sort_temp_bytes(int64_t n);
// Stable LSD sort of keys_in[0,n) (only the low nbits bits are significant);
// writes the sorted keys and the permutation (source index of each output).
void radix_sort(const uint32_t *keys_in, uint32_t *keys_out, uint32_t *perm_out,
                int n, int nbits, void *temp, cudaStream_t s);

}  // namespace sph
