// sph_api.cu -- host engine behind the C ABI of include/sph.h.
//
// An engine owns the device arrays of one or more cases (capacity fixed at
// creation), the per-case constant/dynamic tables and the work stream.  One
// Symplectic step (Eq 33-34) is enqueued as
//   NL(state n): sort keys -> reorder + Tait (Eq 28) -> cell table
//   PI(state n) -> dt (Eq 35) + motion (Eq 37) -> predictor
//   NL(state n+1/2) -> PI(state n+1/2) -> corrector -> t += dt
// with three state buffers: X holds the current state (and the half-step
// state in cell order during PI 2), Y the cell-sorted state n, Z the
// half-step state in Y's order.  The corrector writes state n+1 into X in
// place, so every step has the same buffer roles and can be replayed from
// one captured CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sph.h"
#include "sph_internal.cuh"
#include "sph_kernels.cuh"

using namespace sph;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(expr)                                                              \
  do {                                                                              \
    cudaError_t err_ = (expr);                                                      \
    if (err_ != cudaSuccess)                                                        \
      return fail(SPH_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(err_)); \
  } while (0)

struct Grid {
  double origin[3], cs;
  int nc[3], margin;
  int64_t ncells;
};

int make_grid(const sph_case_params &p, Grid &g) {
  if (!(p.h > 0) || !(p.dp > 0) || !(p.rho0 > 0) || !(p.cs0 > 0) || !(p.gamma > 0))
    return fail(SPH_ERR_ARG, "h, dp, rho0, cs0 and gamma must be positive");
  if (p.cell_mode < 0 || p.cell_mode > 2) return fail(SPH_ERR_ARG, "cell_mode must be 0, 1 or 2");
  if (p.ddt_mode < 0 || p.ddt_mode > 2) return fail(SPH_ERR_ARG, "ddt_mode must be 0, 1 or 2");
  if (p.integrator < 0 || p.integrator > 1)
    return fail(SPH_ERR_ARG, "integrator must be 0 (Symplectic) or 1 (Verlet)");
  if (p.verlet_steps < 0) return fail(SPH_ERR_ARG, "verlet_steps must be >= 0");
  if (p.visc_mode < 0 || p.visc_mode > 1)
    return fail(SPH_ERR_ARG, "visc_mode must be 0 (artificial) or 1 (laminar + SPS)");
  if (!(p.nu0 >= 0)) return fail(SPH_ERR_ARG, "nu0 must be >= 0");
  if (p.boundary_mode < 0 || p.boundary_mode > 1)
    return fail(SPH_ERR_ARG, "boundary_mode must be 0 (DBC) or 1 (mDBC)");
  if (p.mdbc_slip < 0 || p.mdbc_slip > 2) return fail(SPH_ERR_ARG, "mdbc_slip must be 0, 1 or 2");
  const double dmin[3] = {p.domain_min.x, p.domain_min.y, p.domain_min.z};
  const double dmax[3] = {p.domain_max.x, p.domain_max.y, p.domain_max.z};
  // cells of 2h, h or 2h/3: the 2h support spans margin = 1, 2 or 3 cells
  g.margin = p.cell_mode + 1;
  g.cs = 2.0 * p.h / g.margin;
  g.ncells = 1;
  for (int k = 0; k < 3; k++) {
    if (!(dmax[k] > dmin[k])) return fail(SPH_ERR_ARG, "domain_max must exceed domain_min");
    g.origin[k] = dmin[k] - g.margin * g.cs;
    double c = std::ceil((dmax[k] - dmin[k]) / g.cs);
    if (c > 1e7) return fail(SPH_ERR_ARG, "domain too large for the cell grid");
    g.nc[k] = 2 * g.margin + (int)c;
    g.ncells *= g.nc[k];
  }
  if (g.ncells > (int64_t(1) << 30)) return fail(SPH_ERR_ARG, "too many cells");
  return SPH_OK;
}

void fill_const(const sph_case_params &p, const sph_particles &parts, const Grid &g,
                uint32_t cellbase, double t_end, int64_t n_fluid, CaseConst &C) {
  std::memset(&C, 0, sizeof(C));
  for (int k = 0; k < 3; k++) C.origin[k] = g.origin[k];
  C.cs = g.cs;
  C.inv_cs = 1.0 / g.cs;
  C.h_d = p.h;
  C.cs0_d = p.cs0;
  C.cfl = p.cfl;
  C.dt_fixed = p.dt_fixed;
  C.dt_min = p.dt_min;
  C.t_end = t_end;
  C.nmot = parts.n_motions;
  for (int m = 0; m < parts.n_motions; m++) {
    const sph_motion &mo = parts.motions[m];
    C.mot_amp[m] = mo.amplitude;
    C.mot_omega[m] = mo.omega;
    C.mot_phase[m] = mo.phase;
    C.mot_axis[m][0] = (float)mo.axis.x;
    C.mot_axis[m][1] = (float)mo.axis.y;
    C.mot_axis[m][2] = (float)mo.axis.z;
  }
  C.nx = g.nc[0];
  C.ny = g.nc[1];
  C.nz = g.nc[2];
  C.margin = g.margin;
  C.cellbase = cellbase;
  C.ddt = p.ddt_mode;
  C.clamp = p.clamp_boundary_rho != 0;
  C.max_out = p.max_out;
  C.verlet_steps = p.verlet_steps > 0 ? p.verlet_steps : 40;
  C.active = 1;
  C.n_fluid = (int32_t)n_fluid;
  C.h = (float)p.h;
  C.csf = (float)g.cs;
  C.r2max = (float)(4.0 * p.h * p.h);
  C.eta2 = (float)p.eta2;
  const double m = p.rho0 * p.dp * p.dp * p.dp;
  C.m_d = m;
  C.m = (float)m;
  C.rho0 = (float)p.rho0;
  C.inv_rho0 = (float)(1.0 / p.rho0);
  C.btait = (float)(p.cs0 * p.cs0 * p.rho0 / p.gamma);
  C.gamma = (float)p.gamma;
  const double kPi = 3.14159265358979323846;
  const double aD = 21.0 / (16.0 * kPi * p.h * p.h * p.h);  // Eq 11, 3-D
  C.cw = (float)(-5.0 * aD / (p.h * p.h));
  C.wk = (float)aD;
  C.list_k = (float)(1.25 * (p.dt_fixed > 0 ? p.dt_fixed : p.cfl * p.h / p.cs0));
  C.half_inv_h = (float)(0.5 / p.h);
  // artificial viscosity only in visc_mode 0; laminar + SPS constants otherwise
  C.kvisc = p.visc_mode == 0 ? (float)(-2.0 * p.alpha * p.cs0 * p.h) : 0.f;
  C.visc = p.visc_mode;
  C.nu0 = (float)p.nu0;
  C.sps_cs2 = (float)(0.12 * p.dp * 0.12 * p.dp);
  C.sps_cl2 = (float)(0.0066 * p.dp * p.dp);
  C.bmode = p.boundary_mode;
  C.mdbc_slip = p.mdbc_slip;
  C.kddt = p.ddt_mode != 0 ? (float)(2.0 * p.delta * p.h * p.cs0) : 0.f;
  C.g[0] = (float)p.gravity.x;
  C.g[1] = (float)p.gravity.y;
  C.g[2] = (float)p.gravity.z;
  C.cs0f = (float)p.cs0;
  C.inv_csf = (float)(1.0 / g.cs);
  C.inv_gamma = (float)(1.0 / p.gamma);
  const double kB = -p.gamma / (p.cs0 * p.cs0);  // -rho0 / B
  C.khyd[0] = (float)(kB * p.gravity.x);
  C.khyd[1] = (float)(kB * p.gravity.y);
  C.khyd[2] = (float)(kB * p.gravity.z);
  const double k = 1.0 / p.gamma;
  C.hyd_c[0] = (float)((k - 1.0) / 2.0);
  C.hyd_c[1] = (float)((k - 2.0) / 3.0);
  C.hyd_c[2] = (float)((k - 3.0) / 4.0);
}

struct Slot {
  bool used = false;
  sph_case_params params{};
  int64_t n = 0, n_fluid = 0;
  uint32_t cellbase = 0;
  int64_t ncells = 0;
  double t_end = 0;
};

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

void sph::set_last_error(const std::string &msg) { g_err = msg; }

struct sph_engine_t {
  cudaStream_t s = nullptr;
  bool own_stream = false;
  sph_alloc_fn alloc = nullptr;
  sph_free_fn freefn = nullptr;
  void *ctx = nullptr;
  std::vector<std::pair<void *, size_t>> allocs;
  int64_t cap_p = 0, cap_cells = 0;
  int cap_cases = 0;
  int nbits = 0;
  int margin = 0;  // shared by all cases (0: not set yet)
  int integrator = 0;  // 0 Symplectic (Eq 33-34), 1 Verlet (Eq 30-31), all cases
  bool ext = false;    // a case uses Eq 19-20 diffusion or laminar + SPS viscosity
  bool sps = false;    // a case uses laminar + SPS viscosity (tau buffers below)
  bool mdbc = false;   // a case uses the modified dynamic boundary condition
  // neighbour list (pi_variant 3-5): list_cap chunk records per target
  bool list_ok = false;
  bool list_wide = false;  // wide records: beyond 2^25 particles (default physics only)
  bool list_wide_needed = false;  // (then always; else as sph_options.wide_records)
  int list_cap = 0;
  int64_t list_ld = 0;
  uint2 *nlist = nullptr;
  uint16_t *ncount = nullptr;
  float4 *posc_ref = nullptr;  // positions at the list's build (pi_variant 5)
  float4 *posc_ref2 = nullptr; //   the same gathered into a rebuild's new order
  bool list_dirty = true;      // the next kept-list step starts with a rebuild event
  bool list_stale = true;      //   in which every case rebuilds (sorted state overwritten)
  ListCtl *ctl = nullptr;      // rebuild request, build count, list check
  uint32_t *rb_tmp = nullptr;  // tile counts of the restricted rebuild's compaction
  cudaStream_t s2 = nullptr;   // captures the bodies of conditional graph nodes
  // pi_variant 5 without a captured step graph: the two guarded parts of a
  // rebuild (sort + reorder + cell table; skin + list) as small graphs
  cudaGraphExec_t rbx[2] = {nullptr, nullptr};
  int64_t rbx_n = -1, rbx_dead = -1, rbx_hw = -1;
  int rbx_key = -1;
  cudaError_t cap_err = cudaSuccess;  // first error while building a conditional node
  bool capturing = false;             // enqueue_step runs under stream capture
  int list_default = 5;               // pi_variant -1 with a list: the kept list
  int64_t builds_seen = 0;            // ctl->builds at the last check_flags
  float4 *tau4 = nullptr;  // (tau/rho) of Eq 25 in sorted order: xx, yy, zz, xy
  float2 *tau2 = nullptr;  //   xz, yz
  bool pool = false;
  std::vector<Slot> slots;
  std::vector<CaseConst> hconst;
  std::vector<std::pair<int64_t, int64_t>> free_cells;  // [begin, end) ranges
  int64_t n_phys = 0, n_dead = 0;
  int64_t cells_hw = 0;  // cells in use: [0, cells_hw) holds every live case's grid
  // device
  CaseConst *dconst = nullptr;
  CaseDyn *ddyn = nullptr;
  State S[3]{};
  uint32_t *keysA = nullptr, *keysB = nullptr, *keysC = nullptr, *keysD = nullptr;
  uint32_t *perm1 = nullptr, *perm2 = nullptr;
  float4 *ace = nullptr;
  float *mu = nullptr;
  uint32_t *cstart = nullptr;  // cell start table, 2 * (cap_cells + 1) words
  uint32_t *cells_tmp = nullptr;
  float *press = nullptr;
  int *nvalid = nullptr;
  void *sort_tmp = nullptr;
  double *diag = nullptr;
  char *io = nullptr;
  size_t io_bytes = 0;
  // options, graph, timing
  sph_options opt{0, 0, 0, 0, -1.f, 0, 0, 0, 0};  // list_skin < 0: the default
  // pair_once: per-particle sums of the pair-once walk (allocated on first use)
  float4 *sym_sum = nullptr;
  unsigned *sym_mu = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_n = -1, graph_dead = -1;  // n_phys and cells_hw of the captured graph
  int graph_ext = 0;  // ext + 2 sps + 4 mdbc + 8 list of the captured graph
  std::vector<cudaEvent_t> evs;
  double pi_ms = 0, step_ms = 0;
  std::vector<float> step_times;  // per timed step (ms), at most kMaxStepTimes
  int64_t pi_launches = 0, kernel_launches = 0;

  void *dalloc(size_t bytes) {
    bytes = align256(bytes ? bytes : 256);
    void *p = nullptr;
    if (alloc) {
      p = alloc(bytes, (void *)s, ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
    }
    if (p) allocs.push_back({p, bytes});
    return p;
  }
  void drop_graphs() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    for (auto &g : rbx) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
  }
  void release_all() {
    drop_graphs();
    if (s2) cudaStreamDestroy(s2);
    s2 = nullptr;
    for (auto &e : evs) cudaEventDestroy(e);
    evs.clear();
    if (s) cudaStreamSynchronize(s);
    for (auto &a : allocs) {
      if (freefn)
        freefn(a.first, a.second, (void *)s, ctx);
      else
        cudaFree(a.first);
    }
    allocs.clear();
    if (own_stream && s) cudaStreamDestroy(s);
    s = nullptr;
  }
};

namespace {

int bits_for(int64_t cap_cells) { return key_bits(cap_cells); }

// Chunk records a target's list may need (the list segment per target):
// for target offsets sampled over a cell, the rows (dy, dz) whose slab lies
// within R = 2h + skin, each row's cell range in x times ~1.3 (cs/dp)^3
// particles in chunks of 32, plus one record per row for the second
// particle type; x 1.2, rounded up to a multiple of 32.  skin: the largest
// list kept across steps (kListExtraMax x 2h) plus 0.1 h for one step.
constexpr double kListExtraMax = 0.25;
constexpr int64_t kMaxStepTimes = 1 << 20;  // per-step times kept between timing resets

double slab_gap_h(int d, double o, double cs) {
  return d > 0 ? d * cs - o : (d < 0 ? o - (d + 1) * cs : 0.0);
}

int list_records_needed(int cell_mode, double h, double dp) {
  const int M = cell_mode + 1, MR = M + 1;
  const double cs = 2.0 * h / M, R = 2.0 * h + kListExtraMax * 2.0 * h + 0.1 * h;
  const double ppc = 1.3 * std::pow(cs / dp, 3.0);
  const int S = 6;
  double worst = 0.0;
  for (int a = 0; a <= S; a++)
    for (int b = 0; b <= S; b++)
      for (int c = 0; c <= S; c++) {
        const double ox = std::min(a / (double)S, 0.9999) * cs;
        const double oy = std::min(b / (double)S, 0.9999) * cs;
        const double oz = std::min(c / (double)S, 0.9999) * cs;
        double rec = 0.0;
        for (int dy = -MR; dy <= MR; dy++)
          for (int dz = -MR; dz <= MR; dz++) {
            const double gy = slab_gap_h(dy, oy, cs), gz = slab_gap_h(dz, oz, cs);
            const double d2 = gy * gy + gz * gz;
            if (d2 >= R * R) continue;
            const double L = std::sqrt(R * R - d2);
            const int kx0 = std::max(-MR, (int)std::floor((ox - L) / cs));
            const int kx1 = std::min(MR, (int)std::floor((ox + L) / cs));
            rec += std::ceil((kx1 - kx0 + 1) * ppc / 32.0) + 1.0;
          }
        worst = std::max(worst, rec);
      }
  return std::min(4096, ((int)std::ceil(1.2 * worst) + 31) / 32 * 32);
}

// A neighbour list applies to this step: a list variant chosen (3, 4: one
// list per Symplectic step; 5: kept across steps, either scheme) and the
// list allocated.
bool use_list(sph_engine e) {
  if (!e->list_ok) return false;
  if (e->integrator == 1) return e->opt.pi_variant == 5;  // Verlet: one PI per step
  return e->opt.pi_variant >= 3 && e->opt.pi_variant <= 5;
}

// pi_variant as the engine runs it: -1 takes the engine's default; list
// variants fall back to the compacted loop (0) where no list applies (no
// list allocated, or 3 and 4 with the Verlet scheme).
// The pair-once list walk applies: asked for, a list walk, default physics.
// (Variants 4 and 5, whose lists are built alone and can be half lists.  A
// pool's admission that turns it off makes every case build whole lists.)
bool sym_on(sph_engine e) {
  return e->opt.pair_once && e->sym_sum && use_list(e) && e->opt.pi_variant != 3 && !e->ext &&
         !e->sps && !e->mdbc;
}

int resolve_variant(sph_engine e, int v) {
  if (v == -1) v = e->list_ok ? e->list_default : 0;
  if (v == 3 && e->list_wide) v = 4;  // variant 3's records are narrow
  if (v >= 3 && v <= 5 && (!e->list_ok || (e->integrator == 1 && v != 5))) v = 0;
  return v;
}

// The half-step state of the list path: positions and velocity-density of
// z, everything else (case, code, ghost offsets) of y, same order.
State half_state(const State &y, const State &z) {
  State h = y;
  h.posc = z.posc;
  h.velrho = z.velrho;
  return h;
}

// Key of a captured step graph: everything that changes its launches.
int graph_key(sph_engine e) {
  return (int)e->ext + 2 * (int)e->sps + 4 * (int)e->mdbc +
         8 * (use_list(e) ? e->opt.pi_variant - 2 : 0) + 64 * (e->opt.check_list != 0) +
         128 * (int)sym_on(e);
}

int allocate(sph_engine e) {
  const int64_t N = e->cap_p > 0 ? e->cap_p : 1;
  bool ok = true;
  auto A = [&](size_t bytes) {
    void *p = e->dalloc(bytes);
    if (!p) ok = false;
    return p;
  };
  e->dconst = (CaseConst *)A(sizeof(CaseConst) * e->cap_cases);
  e->ddyn = (CaseDyn *)A(sizeof(CaseDyn) * e->cap_cases);
  // kReadPad readable entries past the last particle (interaction reads)
  const int64_t NP = N + kReadPad;
  for (int b = 0; b < 3; b++) {
    e->S[b].posc = (float4 *)A(16 * NP);
    e->S[b].velrho = (float4 *)A(16 * NP);
    e->S[b].id = (uint32_t *)A(4 * N);
    e->S[b].cid = (uint16_t *)A(2 * N);
    e->S[b].code = (uint8_t *)A(N);
    e->S[b].vrprev = e->integrator == 1 && b < 2 ? (float4 *)A(16 * N) : nullptr;
    e->S[b].ghost = e->mdbc || e->pool ? (float4 *)A(16 * N) : nullptr;
  }
  e->keysA = (uint32_t *)A(4 * N);
  e->keysB = (uint32_t *)A(4 * N);
  e->keysC = (uint32_t *)A(4 * N);
  e->keysD = (uint32_t *)A(4 * N);
  e->perm1 = (uint32_t *)A(4 * N);
  e->perm2 = (uint32_t *)A(4 * N);
  e->ace = (float4 *)A(16 * N);
  e->mu = (float *)A(4 * N);
  e->cstart = (uint32_t *)A(4 * (2 * e->cap_cells + 2));
  e->cells_tmp = (uint32_t *)A(4 * cells_temp_words(e->cap_cells));
  e->press = (float *)A(4 * NP);
  if (e->list_ok) {
    e->list_ld = N;
    e->nlist = (uint2 *)A(sizeof(uint2) * (size_t)e->list_cap * (size_t)N);
    e->ncount = (uint16_t *)A(2 * N);
    e->posc_ref = (float4 *)A(16 * N);
    e->posc_ref2 = (float4 *)A(16 * N);
    e->ctl = (ListCtl *)A(sizeof(ListCtl));
    e->rb_tmp = (uint32_t *)A(4 * rb_temp_words(N));
  }
  if (e->sps || e->pool) {
    e->tau4 = (float4 *)A(16 * N);
    e->tau2 = (float2 *)A(8 * N);
  }
  e->nvalid = (int *)A(16);
  e->sort_tmp = A(radix_sort_temp_bytes(N));
  e->diag = (double *)A(sizeof(double) * (8 * 1024 + 8));
  e->io_bytes = align256(64 * (size_t)N) + 4096;
  e->io = (char *)A(e->io_bytes);
  if (!ok) return fail(SPH_ERR_OOM, "device allocation failed");
  for (int b = 0; b < 3; b++) {  // defined contents for the padding
    CUDA_TRY(cudaMemsetAsync(e->S[b].posc, 0, 16 * NP, e->s));
    CUDA_TRY(cudaMemsetAsync(e->S[b].velrho, 0, 16 * NP, e->s));
  }
  CUDA_TRY(cudaMemsetAsync(e->press, 0, 4 * NP, e->s));
  CUDA_TRY(cudaMemsetAsync(e->ddyn, 0, sizeof(CaseDyn) * e->cap_cases, e->s));
  if (e->ctl) CUDA_TRY(cudaMemsetAsync(e->ctl, 0, sizeof(ListCtl), e->s));
  CUDA_TRY(cudaMemsetAsync(e->dconst, 0, sizeof(CaseConst) * e->cap_cases, e->s));
  return SPH_OK;
}

int init_engine(sph_engine e, void *stream, sph_alloc_fn alloc, sph_free_fn freefn, void *ctx) {
  e->alloc = alloc;
  e->freefn = freefn;
  e->ctx = ctx;
  if (stream) {
    e->s = (cudaStream_t)stream;
  } else {
    CUDA_TRY(cudaStreamCreateWithFlags(&e->s, cudaStreamNonBlocking));
    e->own_stream = true;
  }
  return SPH_OK;
}

int check_particles(const sph_case_params *p, const sph_particles *parts) {
  if (!p || !parts) return fail(SPH_ERR_ARG, "null params or particles");
  if (parts->n < 0 || parts->n > (int64_t(1) << 30)) return fail(SPH_ERR_ARG, "bad particle count");
  if (parts->n > 0 && (!parts->pos || !parts->rho || !parts->type))
    return fail(SPH_ERR_ARG, "pos, rho and type are required");
  if (parts->n_motions < 0 || parts->n_motions > kMaxMotions)
    return fail(SPH_ERR_ARG, "at most 8 motions per case");
  if (parts->n_motions > 0 && !parts->motions) return fail(SPH_ERR_ARG, "motions pointer is null");
  if (parts->motion_group)
    for (int64_t i = 0; i < parts->n; i++)
      if (parts->motion_group[i] >= parts->n_motions)
        return fail(SPH_ERR_ARG, "motion_group index out of range");
  if (!(p->cfl > 0) && !(p->dt_fixed > 0)) return fail(SPH_ERR_ARG, "cfl or dt_fixed must be > 0");
  if (p->boundary_mode == 1 && !parts->ghost)
    for (int64_t i = 0; i < parts->n; i++)
      if (parts->type[i] != 0) return fail(SPH_ERR_ARG, "mDBC needs the ghost offsets");
  return SPH_OK;
}

// Copy one case's particles into the device arrays at offset dst0 (slot).
int upload_case(sph_engine e, int slot, const sph_particles *parts, int64_t dst0) {
  const int64_t n = parts->n;
  if (n == 0) return SPH_OK;
  char *p = e->io;
  double *d_pos = (double *)p;
  p += align256(24 * n);
  float *d_vel = (float *)p;
  p += align256(12 * n);
  float *d_rho = (float *)p;
  p += align256(4 * n);
  uint8_t *d_type = (uint8_t *)p;
  p += align256(n);
  int32_t *d_group = (int32_t *)p;
  p += align256(4 * n);
  float *d_ghost = (float *)p;
  CUDA_TRY(cudaMemcpyAsync(d_pos, parts->pos, 24 * n, cudaMemcpyHostToDevice, e->s));
  if (parts->ghost)
    CUDA_TRY(cudaMemcpyAsync(d_ghost, parts->ghost, 12 * n, cudaMemcpyHostToDevice, e->s));
  if (parts->vel) CUDA_TRY(cudaMemcpyAsync(d_vel, parts->vel, 12 * n, cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(cudaMemcpyAsync(d_rho, parts->rho, 4 * n, cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(cudaMemcpyAsync(d_type, parts->type, n, cudaMemcpyHostToDevice, e->s));
  if (parts->motion_group)
    CUDA_TRY(cudaMemcpyAsync(d_group, parts->motion_group, 4 * n, cudaMemcpyHostToDevice, e->s));
  launch_upload((int)n, d_pos, parts->vel ? d_vel : nullptr, d_rho, d_type,
                parts->motion_group ? d_group : nullptr, slot, 0, e->dconst, e->ddyn, e->nbits,
                e->S[0], e->keysA, (int)dst0, parts->ghost ? d_ghost : nullptr, e->s);
  CUDA_TRY(cudaGetLastError());
  // the io buffer is reused by the next call: wait for the copies
  CUDA_TRY(cudaStreamSynchronize(e->s));
  return SPH_OK;
}

int set_slot(sph_engine e, int slot, const sph_case_params *p, const sph_particles *parts,
             const Grid &g, uint32_t cellbase, double t_end) {
  int64_t nf = 0;
  for (int64_t i = 0; i < parts->n; i++) nf += parts->type[i] == 0;
  Slot &S = e->slots[slot];
  S.used = true;
  S.params = *p;
  S.n = parts->n;
  S.n_fluid = nf;
  S.cellbase = cellbase;
  S.ncells = g.ncells;
  S.t_end = t_end;
  fill_const(*p, *parts, g, cellbase, t_end, nf, e->hconst[slot]);
  CUDA_TRY(cudaMemcpyAsync(e->dconst + slot, &e->hconst[slot], sizeof(CaseConst),
                           cudaMemcpyHostToDevice, e->s));
  CaseDyn d;
  std::memset(&d, 0, sizeof(d));
  d.dtmin_bits = kFloatInfBits;
  d.need = 1u;  // a new case builds its list
  CUDA_TRY(cudaMemcpyAsync(e->ddyn + slot, &d, sizeof(CaseDyn), cudaMemcpyHostToDevice, e->s));
  e->list_dirty = true;
  CUDA_TRY(cudaStreamSynchronize(e->s));
  return SPH_OK;
}

// Build an engine holding ncases cases back to back.
int create_engine(const sph_case_params *params, const sph_particles *parts, int ncases,
                  void *stream, sph_alloc_fn alloc, sph_free_fn freefn, void *ctx,
                  sph_engine *out) {
  if (!out) return fail(SPH_ERR_ARG, "null output handle");
  *out = nullptr;
  if (ncases <= 0 || ncases > 65535) return fail(SPH_ERR_ARG, "ncases must be in [1, 65535]");
  std::vector<Grid> grids(ncases);
  int64_t np = 0, nc = 0;
  int margin = 0;
  for (int c = 0; c < ncases; c++) {
    int rc = check_particles(params + c, parts + c);
    if (rc) return rc;
    rc = make_grid(params[c], grids[c]);
    if (rc) return rc;
    if (margin && grids[c].margin != margin)
      return fail(SPH_ERR_ARG, "all cases of an engine must use the same cell_mode");
    if (params[c].integrator != params[0].integrator)
      return fail(SPH_ERR_ARG, "all cases of an engine must use the same integrator");
    margin = grids[c].margin;
    np += parts[c].n;
    nc += grids[c].ncells;
  }
  if (np > (int64_t(1) << 31) - 1) return fail(SPH_ERR_ARG, "too many particles");
  if (nc > (int64_t(1) << 30)) return fail(SPH_ERR_ARG, "too many cells");
  sph_engine e = new sph_engine_t();
  int rc = init_engine(e, stream, alloc, freefn, ctx);
  if (rc) {
    delete e;
    return rc;
  }
  e->cap_p = np;
  e->cap_cells = nc;
  e->cap_cases = ncases;
  e->nbits = bits_for(nc);
  e->margin = margin;
  e->slots.resize(ncases);
  e->hconst.resize(ncases);
  e->integrator = params[0].integrator;
  for (int c = 0; c < ncases; c++) {
    e->ext = e->ext || params[c].ddt_mode == 2 || params[c].visc_mode == 1;
    e->sps = e->sps || params[c].visc_mode == 1;
    e->mdbc = e->mdbc || params[c].boundary_mode == 1;
  }
  // the neighbour list serves every physics option (the Verlet scheme only
  // with the list kept across steps); beyond 2^25 particles its records are
  // wide (the default physics only: the other walks keep the narrow form)
  e->list_ok = np < kListMaxParticles;
  if (!e->list_ok && !e->ext && !e->sps && !e->mdbc && np < ((int64_t)1 << 31)) {
    e->list_ok = true;
    e->list_wide = e->list_wide_needed = true;
  }
  if (e->list_ok) {
    int cap = 32;
    for (int c = 0; c < ncases; c++)
      cap = std::max(cap, list_records_needed(params[c].cell_mode, params[c].h, params[c].dp));
    e->list_cap = cap;
    // the list kept across steps (one list per step, 4, makes every case of a
    // batch take the same steps as alone, bit for bit)
    e->list_default = 5;
  }
  e->opt.pi_variant = resolve_variant(e, -1);
  rc = allocate(e);
  int64_t cell0 = 0, p0 = 0;
  for (int c = 0; c < ncases && rc == SPH_OK; c++) {
    rc = set_slot(e, c, params + c, parts + c, grids[c], (uint32_t)cell0, 0.0);
    if (rc == SPH_OK) rc = upload_case(e, c, parts + c, p0);
    cell0 += grids[c].ncells;
    p0 += parts[c].n;
  }
  if (rc) {
    e->release_all();
    delete e;
    return rc;
  }
  e->n_phys = np;
  e->cells_hw = nc;
  *out = e;
  return SPH_OK;
}

// One Verlet step (all cases): NL and PI on state n, time step, update to
// n+1 written back in X (sorted order).  ev: 2 events around the PI launch.
void enqueue_step_verlet(sph_engine e, cudaEvent_t *ev) {
  const int n = (int)e->n_phys;
  const int nl = (int)(e->n_phys - e->n_dead);
  State &X = e->S[0], &Y = e->S[1];
  cudaStream_t s = e->s;
  radix_sort(e->keysA, e->keysB, e->perm1, n, e->nbits, e->sort_tmp, s);
  launch_reorder(nl, e->perm1, e->keysB, X.posc, X.velrho, X.id, X.cid, X.code, X.vrprev,
                 X.ghost, Y,
                 e->press, e->dconst, e->ddyn, e->nbits, s);
  launch_cells(nl, e->keysB, e->cstart, e->cells_hw, e->nbits, e->nvalid, e->cells_tmp, s);
  if (e->mdbc)
    launch_mdbc(e->margin, nl, e->nvalid, e->keysB, Y, e->press, e->cstart, e->nbits, e->dconst,
                e->ddyn, 0, s);
  if (ev) cudaEventRecord(ev[0], s);
  launch_interact(e->margin, e->opt.pi_variant, nl, e->nvalid, e->keysB, Y.posc, Y.velrho,
                  e->press, Y.cid, e->cstart, e->cells_hw, e->nbits, e->dconst, e->ddyn, e->ace,
                  nullptr, 1, e->ext, e->sps ? e->tau4 : nullptr, e->tau2, s);
  if (ev) cudaEventRecord(ev[1], s);
  launch_dt(e->cap_cases, e->dconst, e->ddyn, s);
  launch_verlet(nl, e->keysB, Y, e->ace, e->dconst, e->ddyn, e->nbits, X, e->keysA, s);
  launch_end_step(e->cap_cases, e->dconst, e->ddyn, s);
}

// The sort of a per-step neighbour list (pi_variant 3, 4): NL on state n
// (X -> Y) with the cell table, and the Eq 38-39 boundary values on it.
void enqueue_list_nl(sph_engine e) {
  const int n = (int)e->n_phys;
  const int nl = (int)(e->n_phys - e->n_dead);
  State &X = e->S[0], &Y = e->S[1];
  cudaStream_t s = e->s;
  radix_sort(e->keysA, e->keysB, e->perm1, n, e->nbits, e->sort_tmp, s);
  launch_reorder(nl, e->perm1, e->keysB, X.posc, X.velrho, X.id, X.cid, X.code, X.vrprev,
                 X.ghost, Y, e->press, e->dconst, e->ddyn, e->nbits, s);
  launch_cells(nl, e->keysB, e->cstart, e->cells_hw, e->nbits, e->nvalid, e->cells_tmp, s);
  if (e->mdbc)  // boundary values of Eq 38-39 on state n
    launch_mdbc(e->margin, nl, e->nvalid, e->keysB, Y, e->press, e->cstart, e->nbits, e->dconst,
                e->ddyn, 0, s);
}

// The first evaluation of a list step, on state n (Y, keysB): pi_variant 4
// builds the list alone and walks it, 3 writes it during a compacted
// evaluation, 5 walks the kept list (its Eq 38-39 boundary values first, in
// the build's cells).  ev: events 0 and 1 (variant 5 records event 0 in its
// guarded rebuild); mu (or null) receives mu_max of Eq 35 per particle.
void enqueue_list_first(sph_engine e, cudaEvent_t *ev, float *mu) {
  const int nl = (int)(e->n_phys - e->n_dead);
  State &Y = e->S[1];
  cudaStream_t s = e->s;
  float4 *tau4 = e->sps ? e->tau4 : nullptr;
  if (e->opt.pi_variant == 5) {
    if (e->mdbc)  // boundary values of Eq 38-39 on state n (the build's cells)
      launch_mdbc(e->margin, nl, e->nvalid, e->keysB, Y, e->press, e->cstart, e->nbits,
                  e->dconst, e->ddyn, 0, s, true);
    launch_interact_list(nl, e->nvalid, e->keysB, Y.posc, Y.velrho, e->press, Y.cid, e->cstart,
                         e->cells_hw, e->nbits, e->dconst, e->ddyn, e->ace, 1, e->nlist,
                         e->list_cap, e->ncount, e->ext, tau4, e->tau2, s, mu,
                         e->opt.pi_block, e->opt.pi_lanes,
                         sym_on(e) ? e->sym_sum : nullptr, e->sym_mu,
                         e->list_wide ? e->keysB : nullptr);
  } else if (e->opt.pi_variant == 4) {  // list alone, then both evaluations over it
    if (ev) cudaEventRecord(ev[0], s);  // the first evaluation's time includes the list
    launch_list_begin(e->cap_cases, e->dconst, e->ddyn, e->ctl, 0.f, 1, e->cstart, e->cells_hw,
                      s);
    launch_build_list(e->margin, nl, e->nvalid, e->keysB, Y.posc, Y.velrho, e->press, Y.cid,
                      e->cstart, e->cells_hw, e->nbits, e->dconst, e->ddyn, e->ace, e->nlist,
                      e->list_cap, e->ncount, nullptr, nullptr, s, sym_on(e), e->list_wide);
    launch_interact_list(nl, e->nvalid, e->keysB, Y.posc, Y.velrho, e->press, Y.cid, e->cstart,
                         e->cells_hw, e->nbits, e->dconst, e->ddyn, e->ace, 1, e->nlist,
                         e->list_cap, e->ncount, e->ext, tau4, e->tau2, s, mu,
                         e->opt.pi_block, e->opt.pi_lanes,
                         sym_on(e) ? e->sym_sum : nullptr, e->sym_mu,
                         e->list_wide ? e->keysB : nullptr);
  } else {
    launch_list_begin(e->cap_cases, e->dconst, e->ddyn, e->ctl, 0.f, 1, e->cstart, e->cells_hw,
                      s);
    if (ev) cudaEventRecord(ev[0], s);
    launch_interact_build(e->margin, nl, e->nvalid, e->keysB, Y.posc, Y.velrho, e->press, Y.cid,
                          e->cstart, e->cells_hw, e->nbits, e->dconst, e->ddyn, e->ace,
                          e->nlist, e->list_cap, e->ncount, e->ext, tau4, e->tau2, s,
                          mu);
  }
  if (ev) cudaEventRecord(ev[1], s);
  if (e->opt.check_list)
    launch_list_check(nl, e->nvalid, e->keysB, Y.posc, Y.cid, e->dconst, e->nbits, e->nlist,
                      e->list_cap, e->ncount, e->ctl, s, sym_on(e),
                      e->list_wide ? e->keysB : nullptr);
}

// The rest of a list step up to its second evaluation: dt (Eq 35), the half
// step into Z in Y's order and cells (Eq 33-34; with the kept list checked
// against the build positions), the Eq 38-39 boundary values on it, and the
// interaction over the list on state n+1/2 (keysC).  ev: events 2 and 3.
void enqueue_list_half(sph_engine e, cudaEvent_t *ev, float *mu) {
  const int nl = (int)(e->n_phys - e->n_dead);
  State &Y = e->S[1], &Z = e->S[2];
  cudaStream_t s = e->s;
  launch_dt(e->cap_cases, e->dconst, e->ddyn, s);
  launch_predictor_list(nl, e->keysB, Y, e->ace, e->dconst, e->ddyn, e->nbits, Z.posc, Z.velrho,
                        e->keysC, e->press, e->opt.pi_variant == 5 ? e->posc_ref : nullptr, s);
  if (e->mdbc)  // boundary values of Eq 38-39 on state n+1/2 (Y's cells)
    launch_mdbc(e->margin, nl, e->nvalid, e->keysC, half_state(Y, Z), e->press, e->cstart,
                e->nbits, e->dconst, e->ddyn, 1, s, true);
  if (ev) cudaEventRecord(ev[2], s);
  launch_interact_list(nl, e->nvalid, e->keysC, Z.posc, Z.velrho, e->press, Y.cid, e->cstart,
                       e->cells_hw, e->nbits, e->dconst, e->ddyn, e->ace, 0, e->nlist,
                       e->list_cap, e->ncount, e->ext, e->sps ? e->tau4 : nullptr, e->tau2, s,
                       mu, e->opt.pi_block, e->opt.pi_lanes,
                         sym_on(e) ? e->sym_sum : nullptr, e->sym_mu,
                         e->list_wide ? e->keysB : nullptr);
  if (ev) cudaEventRecord(ev[3], s);
  if (e->opt.check_list)
    launch_list_check(nl, e->nvalid, e->keysC, Z.posc, Y.cid, e->dconst, e->nbits, e->nlist,
                      e->list_cap, e->ncount, e->ctl, s, sym_on(e),
                      e->list_wide ? e->keysB : nullptr);
}

// One Symplectic step with the per-step neighbour list: NL on state n (Y),
// the list (written by the first PI, variant 3, or built alone and then
// evaluated, variant 4), dt, half step in Y's order and cells (Z), PI over the
// list, full step into X.  ev: 4 events around the two evaluations.
void enqueue_step_list(sph_engine e, cudaEvent_t *ev) {
  const int nl = (int)(e->n_phys - e->n_dead);
  State &X = e->S[0], &Y = e->S[1], &Z = e->S[2];
  enqueue_list_nl(e);
  enqueue_list_first(e, ev, nullptr);
  enqueue_list_half(e, ev, nullptr);
  launch_corrector_list(nl, e->keysB, e->keysC, Y, Z.velrho, e->ace, e->dconst, e->ddyn,
                        e->nbits, X, e->keysA, e->s);
  launch_end_step(e->cap_cases, e->dconst, e->ddyn, e->s);
}

// The two guarded parts of a kept-list rebuild event.  The sort: when index
// ranges may move (ListCtl::full) every particle, the cases that need no
// rebuild entering it with their build keys and build-cell state (so their
// order and cells stay), the others with the normalised state in X; else
// only the particles of the cases that need a rebuild, within their own
// index ranges, the others left untouched in Y.  The build positions follow
// the moved particles.  (An engine of one case sorts directly: its rebuilds
// always involve all its particles.)  Then the cell table of the whole order.
void enqueue_rebuild_sort(sph_engine e, cudaStream_t q) {
  const int n = (int)e->n_phys;
  const int nl = (int)(e->n_phys - e->n_dead);
  State &X = e->S[0], &Y = e->S[1];
  if (e->cap_cases == 1) {
    // one case: every rebuild event sorts all its particles, directly
    radix_sort(e->keysA, e->keysB, e->perm1, n, e->nbits, e->sort_tmp, q);
    launch_reorder(nl, e->perm1, e->keysB, X.posc, X.velrho, X.id, X.cid, X.code, X.vrprev,
                   X.ghost, Y, e->press, e->dconst, e->ddyn, e->nbits, q, e->posc_ref,
                   e->posc_ref2);
  } else {
    launch_select(n, X.cid, e->dconst, e->ddyn, e->keysB, Y.posc, e->keysA, X.posc, e->ctl, q);
    launch_rebuild_sort(n, e->ctl, e->keysA, X, Y, e->keysB, e->press, e->dconst, e->ddyn,
                        e->nbits, e->posc_ref, e->posc_ref2, e->rb_tmp, e->perm2, e->keysC,
                        e->keysD, e->perm1, e->sort_tmp, q);
  }
  launch_cells(nl, e->keysB, e->cstart, e->cells_hw, e->nbits, e->nvalid, e->cells_tmp, q);
}

// The list: per-case skin and build mode, then the build (a case that needs
// it from its state, one whose indices moved from its build positions, the
// rest keep their records).
void enqueue_rebuild_list(sph_engine e, float extra, cudaStream_t q) {
  const int nl = (int)(e->n_phys - e->n_dead);
  State &Y = e->S[1];
  launch_list_begin(e->cap_cases, e->dconst, e->ddyn, e->ctl, extra, 0, e->cstart, e->cells_hw,
                    q);
  launch_build_list(e->margin, nl, e->nvalid, e->keysB, Y.posc, Y.velrho, e->press, Y.cid,
                    e->cstart, e->cells_hw, e->nbits, e->dconst, e->ddyn, e->ace, e->nlist,
                    e->list_cap, e->ncount, e->posc_ref, e->posc_ref2, q, sym_on(e),
                    e->list_wide);
}

// Appends to the graph being captured on e->s a k_decide kernel and an IF
// node whose body (fn's launches, captured on e->s2) runs only while a
// rebuild of the neighbour list is requested (ListCtl::rebuild).
template <class F>
void capture_if_rebuild(sph_engine e, F fn) {
  if (e->cap_err != cudaSuccess) return;
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaGraphConditionalHandle h{};
  cudaGraphNodeParams p{};
  cudaGraphNode_t node{};
  cudaError_t err = cudaStreamGetCaptureInfo(e->s, &st, nullptr, &g, &deps, nullptr, &nd);
  if (!err && st != cudaStreamCaptureStatusActive) err = cudaErrorStreamCaptureInvalidated;
  if (!err) err = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
  if (!err) {
    launch_decide(h, e->ctl, e->s);
    err = cudaStreamGetCaptureInfo(e->s, &st, nullptr, &g, &deps, nullptr, &nd);
  }
  if (!err) {
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    err = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
  }
  if (!err)
    err = cudaStreamUpdateCaptureDependencies(e->s, &node, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
  if (!err)
    err = cudaStreamBeginCaptureToGraph(e->s2, p.conditional.phGraph_out[0], nullptr, nullptr,
                                        0, cudaStreamCaptureModeThreadLocal);
  if (!err) {
    fn(e->s2);
    cudaGraph_t body = nullptr;
    err = cudaStreamEndCapture(e->s2, &body);
  }
  if (err) e->cap_err = err;
}

// The same guarded launches outside a captured step graph: a small graph of
// the decide kernel and the IF node, instantiated once per configuration
// (which: 0 sort + reorder + cell table, 1 skin + list) and launched on e->s.
template <class F>
void eager_if_rebuild(sph_engine e, int which, F fn) {
  if (e->cap_err != cudaSuccess) return;
  const int key = graph_key(e);
  if (e->rbx_n != e->n_phys || e->rbx_dead != e->n_dead || e->rbx_hw != e->cells_hw ||
      e->rbx_key != key) {
    for (auto &x : e->rbx) {
      if (x) cudaGraphExecDestroy(x);
      x = nullptr;
    }
    e->rbx_n = e->n_phys;
    e->rbx_dead = e->n_dead;
    e->rbx_hw = e->cells_hw;
    e->rbx_key = key;
  }
  if (!e->rbx[which]) {
    cudaError_t err = cudaStreamBeginCapture(e->s, cudaStreamCaptureModeThreadLocal);
    if (err) {
      e->cap_err = err;
      return;
    }
    capture_if_rebuild(e, fn);
    cudaGraph_t g = nullptr;
    err = cudaStreamEndCapture(e->s, &g);
    if (!err && e->cap_err == cudaSuccess) err = cudaGraphInstantiate(&e->rbx[which], g, 0);
    if (g) cudaGraphDestroy(g);
    if (err && e->cap_err == cudaSuccess) e->cap_err = err;
    if (e->cap_err != cudaSuccess) return;
  }
  cudaError_t err = cudaGraphLaunch(e->rbx[which], e->s);
  if (err) e->cap_err = err;
}

// The guarded part of a step on the kept list: while a rebuild is requested,
// the sort, reorder and cell table of the current state (X -> Y), then the
// skin and the list on Y with every target's position (posc_ref); as IF nodes
// of the captured step graph, or as small graphs launched eagerly (ev[0]
// then sits between the two parts, so that the first evaluation's time
// includes the list build).
void enqueue_reuse_rebuild(sph_engine e, cudaEvent_t *ev) {
  const float extra = e->opt.list_skin >= 0.f ? e->opt.list_skin : 0.04f;
  auto nl_part = [=](cudaStream_t q) { enqueue_rebuild_sort(e, q); };
  auto list_part = [=](cudaStream_t q) { enqueue_rebuild_list(e, extra, q); };
  if (e->capturing) {
    capture_if_rebuild(e, nl_part);
    capture_if_rebuild(e, list_part);
  } else {
    eager_if_rebuild(e, 0, nl_part);
    if (ev) cudaEventRecord(ev[0], e->s);
    eager_if_rebuild(e, 1, list_part);
  }
}

// One Symplectic step over the neighbour list kept across steps (pi_variant
// 5).  Guarded by the rebuild request: sort, reorder and cell table of the
// current state (X -> Y), then the skin and the list on Y with every target's
// position (posc_ref).  Always: PI on Y (state n), dt, half step into Z in Y's
// order and cells, PI on Z, and the corrector, which writes state n+1 to X
// (normalised, keysA) and in place to Y, and requests a rebuild when the next
// step could leave the skin.  ev: 4 events around the two evaluations (the
// first one's time includes the list build when it runs).
void enqueue_step_reuse(sph_engine e, cudaEvent_t *ev) {
  const int nl = (int)(e->n_phys - e->n_dead);
  State &X = e->S[0], &Y = e->S[1], &Z = e->S[2];
  enqueue_reuse_rebuild(e, ev);
  enqueue_list_first(e, ev, nullptr);
  enqueue_list_half(e, ev, nullptr);
  launch_corrector_reuse(nl, e->keysB, e->keysC, Y, Z.velrho, e->ace, e->posc_ref, e->dconst,
                         e->ddyn, e->nbits, X, e->keysA, e->press, e->ctl, e->s);
  launch_end_step(e->cap_cases, e->dconst, e->ddyn, e->s);
}

// One Verlet step over the list kept across steps: the guarded sort +
// reorder + cell table and skin + list (as enqueue_step_reuse), the PI on Y,
// dt, and the update, which writes state n+1 to X (normalised) and in place to
// Y and requests a rebuild when a particle is farther than (skin - 1e-3 h)/2
// from its build position.  ev: 2 events around the PI (the build included).
void enqueue_step_verlet_reuse(sph_engine e, cudaEvent_t *ev) {
  const int nl = (int)(e->n_phys - e->n_dead);
  State &X = e->S[0], &Y = e->S[1];
  enqueue_reuse_rebuild(e, ev);
  enqueue_list_first(e, ev, nullptr);
  launch_dt(e->cap_cases, e->dconst, e->ddyn, e->s);
  launch_verlet_reuse(nl, e->keysB, Y, e->ace, e->dconst, e->ddyn, e->nbits, X, e->keysA,
                      e->posc_ref, e->press, e->ctl, e->s);
  launch_end_step(e->cap_cases, e->dconst, e->ddyn, e->s);
}

// One Symplectic step (all cases).  ev: 4 events around the two PI launches.
void enqueue_step(sph_engine e, cudaEvent_t *ev) {
  if (e->integrator == 1) {
    if (use_list(e))
      enqueue_step_verlet_reuse(e, ev);
    else
      enqueue_step_verlet(e, ev);
    return;
  }
  if (use_list(e)) {
    if (e->opt.pi_variant == 5)
      enqueue_step_reuse(e, ev);
    else
      enqueue_step_list(e, ev);
    return;
  }
  const int n = (int)e->n_phys;
  const int nl = (int)(e->n_phys - e->n_dead);
  State &X = e->S[0], &Y = e->S[1], &Z = e->S[2];
  cudaStream_t s = e->s;
  // NL on state n
  radix_sort(e->keysA, e->keysB, e->perm1, n, e->nbits, e->sort_tmp, s);
  launch_reorder(nl, e->perm1, e->keysB, X.posc, X.velrho, X.id, X.cid, X.code, X.vrprev,
                 X.ghost, Y,
                 e->press, e->dconst, e->ddyn, e->nbits, s);
  launch_cells(nl, e->keysB, e->cstart, e->cells_hw, e->nbits, e->nvalid, e->cells_tmp, s);
  if (e->mdbc)  // boundary values of Eq 38-39 on state n
    launch_mdbc(e->margin, nl, e->nvalid, e->keysB, Y, e->press, e->cstart, e->nbits, e->dconst,
                e->ddyn, 0, s);
  // PI on state n, time step, predictor
  if (ev) cudaEventRecord(ev[0], s);
  launch_interact(e->margin, e->opt.pi_variant, nl, e->nvalid, e->keysB, Y.posc, Y.velrho,
                  e->press, Y.cid, e->cstart, e->cells_hw, e->nbits, e->dconst, e->ddyn, e->ace,
                  nullptr, 1, e->ext, e->sps ? e->tau4 : nullptr, e->tau2, s);
  if (ev) cudaEventRecord(ev[1], s);
  launch_dt(e->cap_cases, e->dconst, e->ddyn, s);
  launch_predictor(nl, e->keysB, Y, e->ace, e->dconst, e->ddyn, e->nbits, Z.posc, Z.velrho,
                   e->keysC, s);
  // NL on state n+1/2 (id/cid/code of Z are those of Y)
  radix_sort(e->keysC, e->keysD, e->perm2, nl, e->nbits, e->sort_tmp, s);
  launch_reorder(nl, e->perm2, e->keysD, Z.posc, Z.velrho, Y.id, Y.cid, Y.code, nullptr,
                 Y.ghost, X,
                 e->press, e->dconst, e->ddyn, e->nbits, s);
  launch_cells(nl, e->keysD, e->cstart, e->cells_hw, e->nbits, e->nvalid + 1, e->cells_tmp, s);
  if (e->mdbc)  // boundary values of Eq 38-39 on state n+1/2
    launch_mdbc(e->margin, nl, e->nvalid + 1, e->keysD, X, e->press, e->cstart, e->nbits,
                e->dconst, e->ddyn, 1, s);
  if (ev) cudaEventRecord(ev[2], s);
  launch_interact(e->margin, e->opt.pi_variant, nl, e->nvalid + 1, e->keysD, X.posc, X.velrho,
                  e->press, X.cid, e->cstart, e->cells_hw, e->nbits, e->dconst, e->ddyn, e->ace,
                  nullptr, 0, e->ext, e->sps ? e->tau4 : nullptr, e->tau2, s);
  if (ev) cudaEventRecord(ev[3], s);
  launch_corrector(nl, e->perm2, e->keysD, e->keysB, Y, X, e->ace, e->dconst, e->ddyn, e->nbits,
                   e->keysA, s);
  launch_end_step(e->cap_cases, e->dconst, e->ddyn, s);
}

// NL only, on the current state: keysA/X -> keysB/Y + cell table (the kept
// list's sorted state is gone: its next step rebuilds every case).
void enqueue_nl(sph_engine e) {
  e->list_stale = true;
  const int n = (int)e->n_phys;
  const int nl = (int)(e->n_phys - e->n_dead);
  State &X = e->S[0], &Y = e->S[1];
  radix_sort(e->keysA, e->keysB, e->perm1, n, e->nbits, e->sort_tmp, e->s);
  launch_reorder(nl, e->perm1, e->keysB, X.posc, X.velrho, X.id, X.cid, X.code, X.vrprev,
                 X.ghost, Y,
                 e->press,
                 e->dconst, e->ddyn, e->nbits, e->s);
  launch_cells(nl, e->keysB, e->cstart, e->cells_hw, e->nbits, e->nvalid, e->cells_tmp, e->s);
}

int check_flags(sph_engine e) {
  std::vector<CaseDyn> d(e->cap_cases);
  CUDA_TRY(cudaMemcpyAsync(d.data(), e->ddyn, sizeof(CaseDyn) * e->cap_cases,
                           cudaMemcpyDeviceToHost, e->s));
  ListCtl lc{};
  if (e->ctl)
    CUDA_TRY(cudaMemcpyAsync(&lc, e->ctl, sizeof(ListCtl), cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  e->builds_seen = (int64_t)lc.builds;
  for (int c = 0; c < e->cap_cases; c++) {
    if (!e->slots[c].used) continue;
    if (d[c].flags & kFlagNaN)
      return fail(SPH_ERR_UNSTABLE, "case " + std::to_string(c) + ": NaN/Inf in the interaction");
    if (d[c].flags & kFlagDtMin)
      return fail(SPH_ERR_UNSTABLE, "case " + std::to_string(c) + ": dt below dt_min");
    if (d[c].flags & kFlagListFull)
      return fail(SPH_ERR_STATE, "case " + std::to_string(c) +
                                     ": a particle has more neighbour-list candidates than the "
                                     "list holds; use pi_variant 0");
    if (d[c].flags & kFlagSkin)
      return fail(SPH_ERR_UNSTABLE, "case " + std::to_string(c) +
                                        ": a displacement since the neighbour list's build "
                                        "exceeded half its skin, or one step needs a skin the "
                                        "list's rows do not reach; use pi_variant 0");
    int mo = e->hconst[c].max_out;
    if (mo >= 0 && d[c].n_out > mo)
      return fail(SPH_ERR_DOMAIN, "case " + std::to_string(c) + ": " +
                                      std::to_string(d[c].n_out) + " particles left the domain");
  }
  return SPH_OK;
}

int valid_case(sph_engine e, int icase) {
  if (!e) return fail(SPH_ERR_ARG, "null engine");
  if (icase < 0 || icase >= e->cap_cases || !e->slots[icase].used)
    return fail(SPH_ERR_ARG, "no such case");
  return SPH_OK;
}

}  // namespace

// ============================================================================
extern "C" {

const char *sph_last_error(void) { return g_err.c_str(); }

int sph_create(const sph_case_params *params, const sph_particles *parts, void *stream,
               sph_alloc_fn alloc, sph_free_fn free_fn, void *alloc_ctx, sph_engine *out) {
  return create_engine(params, parts, 1, stream, alloc, free_fn, alloc_ctx, out);
}

int sph_batch_create(const sph_case_params *params, const sph_particles *parts, int32_t ncases,
                     void *stream, sph_alloc_fn alloc, sph_free_fn free_fn, void *alloc_ctx,
                     sph_engine *out) {
  if (!params || !parts) return fail(SPH_ERR_ARG, "null params or particles");
  return create_engine(params, parts, ncases, stream, alloc, free_fn, alloc_ctx, out);
}

int sph_set_options(sph_engine e, const sph_options *opt) {
  if (!e || !opt) return fail(SPH_ERR_ARG, "null argument");
  if (opt->pi_block != 0 && opt->pi_block != 128 && opt->pi_block != 256 &&
      opt->pi_block != 512 && opt->pi_block != 1024)
    return fail(SPH_ERR_ARG, "pi_block must be 0 (default), 128, 256, 512 or 1024");
  if (opt->pi_lanes != 0 && opt->pi_lanes != 1 && opt->pi_lanes != 2 && opt->pi_lanes != 4 &&
      opt->pi_lanes != 8)
    return fail(SPH_ERR_ARG, "pi_lanes must be 0 (default), 1, 2, 4 or 8");
  if (opt->pair_once != 0 && opt->pair_once != 1)
    return fail(SPH_ERR_ARG, "pair_once must be 0 or 1");
  if (opt->wide_records != 0 && opt->wide_records != 1)
    return fail(SPH_ERR_ARG, "wide_records must be 0 or 1");
  if (opt->pair_once && !e->sym_sum) {
    const int64_t N = e->cap_p > 0 ? e->cap_p : 1;
    e->sym_sum = (float4 *)e->dalloc(16 * N);
    e->sym_mu = (unsigned *)e->dalloc(4 * N);
    if (!e->sym_sum || !e->sym_mu) return fail(SPH_ERR_OOM, "device allocation failed");
    CUDA_TRY(cudaMemsetAsync(e->sym_sum, 0, 16 * N, e->s));
    CUDA_TRY(cudaMemsetAsync(e->sym_mu, 0, 4 * N, e->s));
  }
  if (opt->pi_variant < -1 || opt->pi_variant > 6)
    return fail(SPH_ERR_ARG,
                "pi_variant must be -1 (engine default), 0 (compacted), 1 (inline), 2 (queued), "
                "3 (per-step list written by the first evaluation), 4 (per-step list built "
                "alone), 5 (list kept across steps) or 6 (warp-shared candidate tiles)");
  if (opt->list_skin > (float)kListExtraMax)
    return fail(SPH_ERR_ARG, "list_skin must be at most 0.25 (or < 0 for the default)");
  e->opt = *opt;
  // wide records where needed, or where asked for and the physics allows them
  e->list_wide = e->list_wide_needed ||
                 (opt->wide_records && e->list_ok && !e->ext && !e->sps && !e->mdbc && !e->pool);
  e->opt.pi_variant = resolve_variant(e, opt->pi_variant);
  e->list_stale = true;  // another pair loop may have run in between
  e->drop_graphs();
  return SPH_OK;
}

int sph_step(sph_engine e, int64_t nsteps) {
  if (!e) return fail(SPH_ERR_ARG, "null engine");
  if (nsteps < 0) return fail(SPH_ERR_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return SPH_OK;
  if (e->n_phys == 0) return SPH_OK;
  const bool timing = e->opt.timing != 0;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (timing) {
    size_t need = 4 * (size_t)nsteps + 2;
    while (e->evs.size() < need) {
      cudaEvent_t ev;
      CUDA_TRY(cudaEventCreate(&ev));
      e->evs.push_back(ev);
    }
    t0 = e->evs[4 * nsteps];
    t1 = e->evs[4 * nsteps + 1];
    CUDA_TRY(cudaEventRecord(t0, e->s));
  }
  int64_t k = 0;
  const bool reuse = use_list(e) && e->opt.pi_variant == 5;
  if (reuse) {
    if (!e->s2) CUDA_TRY(cudaStreamCreateWithFlags(&e->s2, cudaStreamNonBlocking));
    // a call continues the kept list as if the steps had not been split,
    // unless the cases or the sorted state changed since the last step
    if (e->list_stale) launch_need_all(e->cap_cases, e->ddyn, e->s);
    if (e->list_stale || e->list_dirty)  // a rebuild of every case: ranges may have moved
      CUDA_TRY(cudaMemsetAsync(&e->ctl->rebuild, 1, 2 * sizeof(unsigned int), e->s));
    e->list_stale = e->list_dirty = false;
  }
  e->cap_err = cudaSuccess;
  if (!timing && e->opt.use_graph && e->n_dead == 0) {
    if (!e->gexec || e->graph_n != e->n_phys || e->graph_dead != e->cells_hw ||
        e->graph_ext != graph_key(e)) {
      if (e->gexec) cudaGraphExecDestroy(e->gexec);
      e->gexec = nullptr;
      cudaGraph_t g;
      CUDA_TRY(cudaStreamBeginCapture(e->s, cudaStreamCaptureModeThreadLocal));
      e->capturing = true;
      enqueue_step(e, nullptr);
      e->capturing = false;
      cudaError_t err = cudaStreamEndCapture(e->s, &g);
      if (err == cudaSuccess && e->cap_err != cudaSuccess) {
        cudaGraphDestroy(g);
        err = e->cap_err;
      } else if (err == cudaSuccess) {
        err = cudaGraphInstantiate(&e->gexec, g, 0);
        cudaGraphDestroy(g);
      }
      if (err != cudaSuccess) return fail(SPH_ERR_CUDA, cudaGetErrorString(err));
      e->graph_n = e->n_phys;
      e->graph_dead = e->cells_hw;  // cells in use at capture
      e->graph_ext = graph_key(e);
    }
    for (; k < nsteps; k++) CUDA_TRY(cudaGraphLaunch(e->gexec, e->s));
  }
  // per Symplectic step: 2 sorts (3 kernels per 8-bit pass), 2 reorders, 2
  // cell tables (4 kernels), 2 interactions, dt, predictor, corrector, end of
  // step; with the per-step list: one sort, reorder, cell table, the list, 2
  // interactions, dt, predictor, corrector, end; per Verlet step: one sort,
  // reorder, cell table and interaction, dt, update, end of step
  const int64_t passes = std::max(1, (e->nbits + 7) / 8);
  const int64_t pis = e->integrator == 1 ? 1 : 2;
  const bool listed = use_list(e);
  // (the list kept across steps: 2 decide kernels, 2 interactions, dt,
  // predictor, corrector, end per step; the sort, reorder, cell table, skin
  // and list per build, counted from the device's build counter)
  const int64_t per_step = (e->integrator == 1 ? (reuse ? 2 + 1 + 3 : 3 * passes + 1 + 4 + 1 + 3)
                            : reuse            ? 2 + 2 + 4
                            : listed           ? 3 * passes + 1 + 4 + 1 + 2 + 4 +
                                                     (e->opt.pi_variant == 4 ? 1 : 0)
                                               : 6 * passes + 2 + 8 + 2 + 4) +
                           (e->sps ? pis : 0) +  // strain pass before each interaction
                           (e->mdbc ? pis : 0) +  // ghost-node pass before each interaction
                           (listed && e->opt.check_list ? pis : 0) +
                           (sym_on(e) ? pis : 0);  // the pair-once finish
  e->kernel_launches += per_step * nsteps;
  for (; k < nsteps; k++) {
    enqueue_step(e, timing ? &e->evs[4 * k] : nullptr);
    e->n_phys -= e->n_dead;
    e->n_dead = 0;
  }
  if (timing) CUDA_TRY(cudaEventRecord(t1, e->s));
  CUDA_TRY(cudaGetLastError());
  if (e->cap_err != cudaSuccess) {
    cudaStreamSynchronize(e->s);
    return fail(SPH_ERR_CUDA, std::string("conditional graph node: ") +
                                  cudaGetErrorString(e->cap_err));
  }
  CUDA_TRY(cudaStreamSynchronize(e->s));
  if (timing) {
    for (int64_t j = 0; j < nsteps; j++) {
      float a = 0.f, b = 0.f, d = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&a, e->evs[4 * j], e->evs[4 * j + 1]));
      if (e->integrator != 1)
        CUDA_TRY(cudaEventElapsedTime(&b, e->evs[4 * j + 2], e->evs[4 * j + 3]));
      e->pi_ms += a + b;
      e->pi_launches += e->integrator == 1 ? 1 : 2;
      // step j: from the start of its first interaction to the start of the
      // next step's (the call's last step: to the end of the call)
      CUDA_TRY(cudaEventElapsedTime(&d, e->evs[4 * j], j + 1 < nsteps ? e->evs[4 * (j + 1)] : t1));
      if ((int64_t)e->step_times.size() < kMaxStepTimes) e->step_times.push_back(d);
    }
    float tot = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&tot, t0, t1));
    e->step_ms += tot;
  }
  const int64_t builds0 = e->builds_seen;
  const int rc = check_flags(e);
  // per rebuild event: the sort (3 kernels per pass), the reorder (one case) or
  // select + count + scan + compact + scatter (several), the cell table (4),
  // the skin and the list build
  if (reuse)
    e->kernel_launches += (e->builds_seen - builds0) *
                          (3 * passes + (e->cap_cases == 1 ? 1 : 5) + 4 + 1 + 1);
  return rc;
}

int sph_get_timing(sph_engine e, double *pi_ms, int64_t *pi_launches, double *step_ms,
                   int64_t *kernel_launches, int32_t reset) {
  if (!e) return fail(SPH_ERR_ARG, "null engine");
  if (pi_ms) *pi_ms = e->pi_ms;
  if (pi_launches) *pi_launches = e->pi_launches;
  if (step_ms) *step_ms = e->step_ms;
  if (kernel_launches) *kernel_launches = e->kernel_launches;
  if (reset) {
    e->pi_ms = e->step_ms = 0;
    e->pi_launches = 0;
    e->kernel_launches = 0;
    e->step_times.clear();
  }
  return SPH_OK;
}

int sph_get_step_times(sph_engine e, float *ms, int64_t cap, int64_t *n) {
  if (!e) return fail(SPH_ERR_ARG, "null engine");
  if (cap < 0) return fail(SPH_ERR_ARG, "cap must be >= 0");
  const int64_t have = (int64_t)e->step_times.size();
  if (ms && cap > 0) std::copy_n(e->step_times.begin(), std::min(have, cap), ms);
  if (n) *n = have;
  return SPH_OK;
}

int sph_list_info(sph_engine e, int64_t *builds, int64_t *check_pairs, int64_t *check_bad) {
  if (!e) return fail(SPH_ERR_ARG, "null engine");
  ListCtl lc{};
  if (e->ctl) {
    CUDA_TRY(cudaMemcpyAsync(&lc, e->ctl, sizeof(ListCtl), cudaMemcpyDeviceToHost, e->s));
    CUDA_TRY(cudaStreamSynchronize(e->s));
  }
  if (builds) *builds = (int64_t)lc.builds;
  if (check_pairs) *check_pairs = (int64_t)lc.check_pairs;
  if (check_bad) *check_bad = (int64_t)lc.check_bad;
  return SPH_OK;
}

int sph_get_state(sph_engine e, int32_t icase, double *pos, float *vel, float *rho, float *press,
                  double *t, int64_t *step, double *last_dt) {
  int rc = valid_case(e, icase);
  if (rc) return rc;
  const int64_t n = e->slots[icase].n;
  char *p = e->io;
  double *d_pos = (double *)p;
  p += align256(24 * n);
  float *d_vel = (float *)p;
  p += align256(12 * n);
  float *d_rho = (float *)p;
  p += align256(4 * n);
  float *d_press = (float *)p;
  launch_export((int)e->n_phys, e->keysA, e->S[0], e->dconst, icase, 0, e->nbits,
                pos ? d_pos : nullptr, vel ? d_vel : nullptr, rho ? d_rho : nullptr,
                press ? d_press : nullptr, e->s);
  CUDA_TRY(cudaGetLastError());
  if (pos) CUDA_TRY(cudaMemcpyAsync(pos, d_pos, 24 * n, cudaMemcpyDeviceToHost, e->s));
  if (vel) CUDA_TRY(cudaMemcpyAsync(vel, d_vel, 12 * n, cudaMemcpyDeviceToHost, e->s));
  if (rho) CUDA_TRY(cudaMemcpyAsync(rho, d_rho, 4 * n, cudaMemcpyDeviceToHost, e->s));
  if (press) CUDA_TRY(cudaMemcpyAsync(press, d_press, 4 * n, cudaMemcpyDeviceToHost, e->s));
  CaseDyn d;
  CUDA_TRY(cudaMemcpyAsync(&d, e->ddyn + icase, sizeof(d), cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  if (t) *t = d.t;
  if (step) *step = d.step;
  if (last_dt) *last_dt = d.dt;
  return SPH_OK;
}

int sph_get_stats(sph_engine e, int32_t icase, sph_stats *out) {
  int rc = valid_case(e, icase);
  if (rc) return rc;
  if (!out) return fail(SPH_ERR_ARG, "null output");
  const int nparts = 512;
  launch_diag((int)e->n_phys, e->keysA, e->S[0], e->dconst, icase, e->nbits, e->diag + 8, nparts,
              e->diag, e->s);
  CUDA_TRY(cudaGetLastError());
  double v[8];
  CaseDyn d;
  CUDA_TRY(cudaMemcpyAsync(v, e->diag, sizeof(v), cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaMemcpyAsync(&d, e->ddyn + icase, sizeof(d), cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  out->t = d.t;
  out->last_dt = d.dt;
  out->step = d.step;
  out->interactions = (int64_t)d.pairs;
  out->interactions_fb = (int64_t)d.pairs_fb;
  out->interactions_bf = (int64_t)d.pairs_bf;
  out->mass = v[0] * e->hconst[icase].m_d;
  out->kinetic_energy = v[1];
  out->momentum[0] = v[2];
  out->momentum[1] = v[3];
  out->momentum[2] = v[4];
  out->front = v[6];
  out->n_out = (int64_t)v[7];
  out->flags = (int32_t)d.flags;
  out->n_fluid = (int32_t)e->slots[icase].n_fluid;
  out->n = e->slots[icase].n;
  return SPH_OK;
}

// ---- checkpoint ----------------------------------------------------------------

namespace {
struct RawHeader {
  uint32_t magic, version;
  int64_t n;
  double t, dt;
  int64_t step;
  uint64_t pairs;
  int32_t n_out, flags;
};
constexpr uint32_t kRawMagic = 0x52485053u;  // "SPHR"
}  // namespace

int sph_get_raw(sph_engine e, int32_t icase, void *buf, size_t *bytes) {
  int rc = valid_case(e, icase);
  if (rc) return rc;
  if (!bytes) return fail(SPH_ERR_ARG, "null size pointer");
  const int64_t n = e->slots[icase].n;
  const bool verlet = e->integrator == 1;
  const size_t need = sizeof(RawHeader) + (size_t)n * (4 + 4 + 16 + 16 + (verlet ? 16 : 0));
  if (!buf) {
    *bytes = need;
    return SPH_OK;
  }
  if (*bytes < need) return fail(SPH_ERR_ARG, "raw buffer too small");
  *bytes = need;
  // a snapshot holds the normalised state only: the next step rebuilds every
  // case's list, as the first step of an engine resumed from it does
  e->list_stale = true;
  // device order of the case = order in X, filtered by slot (host-side)
  const int64_t np = e->n_phys;
  std::vector<uint32_t> keys(np), ids(np);
  std::vector<uint16_t> cid(np);
  std::vector<float4> pc(np), vr(np), vp(verlet ? np : 0);
  CUDA_TRY(cudaMemcpyAsync(keys.data(), e->keysA, 4 * np, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaMemcpyAsync(ids.data(), e->S[0].id, 4 * np, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaMemcpyAsync(cid.data(), e->S[0].cid, 2 * np, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaMemcpyAsync(pc.data(), e->S[0].posc, 16 * np, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaMemcpyAsync(vr.data(), e->S[0].velrho, 16 * np, cudaMemcpyDeviceToHost, e->s));
  if (verlet)
    CUDA_TRY(cudaMemcpyAsync(vp.data(), e->S[0].vrprev, 16 * np, cudaMemcpyDeviceToHost, e->s));
  CaseDyn d;
  CUDA_TRY(cudaMemcpyAsync(&d, e->ddyn + icase, sizeof(d), cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  RawHeader hd{kRawMagic, verlet ? 2u : 1u, n, d.t, d.dt, d.step, d.pairs, d.n_out,
               (int32_t)d.flags};
  char *o = (char *)buf;
  std::memcpy(o, &hd, sizeof(hd));
  uint32_t *oid = (uint32_t *)(o + sizeof(hd));
  int32_t *ocell = (int32_t *)(oid + n);
  float4 *opc = (float4 *)(ocell + n);
  float4 *ovr = opc + n;
  float4 *ovp = ovr + n;  // version 2 only
  const uint32_t kdead = key_dead(e->nbits), kout = key_out(e->nbits);
  const uint32_t cb = e->slots[icase].cellbase;
  int64_t j = 0;
  for (int64_t i = 0; i < np && j < n; i++) {
    if (cid[i] != icase || keys[i] == kdead) continue;
    oid[j] = ids[i];
    ocell[j] = keys[i] >= kout ? -1 : (int32_t)(key_cell(keys[i], e->nbits) - cb);
    std::memcpy(opc + j, &pc[i], 16);
    std::memcpy(ovr + j, &vr[i], 16);
    if (verlet) std::memcpy(ovp + j, &vp[i], 16);
    j++;
  }
  if (j != n) return fail(SPH_ERR_STATE, "raw export found the wrong particle count");
  return SPH_OK;
}

int sph_create_from_raw(const sph_case_params *params, const sph_particles *parts,
                        const void *buf, size_t bytes, void *stream, sph_alloc_fn alloc,
                        sph_free_fn free_fn, void *alloc_ctx, sph_engine *out) {
  if (!buf || bytes < sizeof(RawHeader)) return fail(SPH_ERR_ARG, "bad raw buffer");
  RawHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kRawMagic || (hd.version != 1 && hd.version != 2))
    return fail(SPH_ERR_ARG, "not a raw snapshot");
  if (!params || (params->integrator == 1) != (hd.version == 2))
    return fail(SPH_ERR_ARG, "snapshot and params disagree on the integrator");
  if (!parts || parts->n != hd.n) return fail(SPH_ERR_ARG, "particle count does not match snapshot");
  if (bytes < sizeof(RawHeader) + (size_t)hd.n * (hd.version == 2 ? 56 : 40))
    return fail(SPH_ERR_ARG, "truncated snapshot");
  int rc = create_engine(params, parts, 1, stream, alloc, free_fn, alloc_ctx, out);
  if (rc) return rc;
  sph_engine e = *out;
  const int64_t n = hd.n;
  const char *o = (const char *)buf + sizeof(hd);
  const uint32_t *ids = (const uint32_t *)o;
  const int32_t *cell = (const int32_t *)(ids + n);
  const float4 *pc = (const float4 *)(cell + n);
  const float4 *vr = pc + n;
  // reorder type/group into snapshot order on the host, then import
  std::vector<uint8_t> type(n);
  std::vector<int32_t> group(n, -1);
  std::vector<float> ghost(parts->ghost ? 3 * n : 0);
  for (int64_t j = 0; j < n; j++) {
    if (ids[j] >= (uint32_t)n) {
      sph_destroy(e);
      *out = nullptr;
      return fail(SPH_ERR_ARG, "bad id in snapshot");
    }
    type[j] = parts->type[ids[j]];
    if (parts->motion_group) group[j] = parts->motion_group[ids[j]];
    if (parts->ghost)
      for (int k = 0; k < 3; k++) ghost[3 * j + k] = parts->ghost[3 * ids[j] + k];
  }
  char *p = e->io;
  int32_t *d_cell = (int32_t *)p;
  p += align256(4 * n);
  float4 *d_pc = (float4 *)p;
  p += align256(16 * n);
  float4 *d_vr = (float4 *)p;
  p += align256(16 * n);
  uint8_t *d_type = (uint8_t *)p;
  p += align256(n);
  int32_t *d_group = (int32_t *)p;
  p += align256(4 * n);
  float *d_ghost = (float *)p;
  if (parts->ghost)
    CUDA_TRY(cudaMemcpyAsync(d_ghost, ghost.data(), 12 * n, cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(cudaMemcpyAsync(d_cell, cell, 4 * n, cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(cudaMemcpyAsync(d_pc, pc, 16 * n, cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(cudaMemcpyAsync(d_vr, vr, 16 * n, cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(cudaMemcpyAsync(d_type, type.data(), n, cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(cudaMemcpyAsync(d_group, group.data(), 4 * n, cudaMemcpyHostToDevice, e->s));
  launch_import_raw((int)n, d_cell, d_pc, d_vr, d_type, d_group, 0, 0, e->dconst, e->nbits,
                    e->S[0], e->keysA, 0, parts->ghost ? d_ghost : nullptr, e->s);
  // ids: the import wrote 0..n-1; restore the snapshot ids
  CUDA_TRY(cudaMemcpyAsync(e->S[0].id, ids, 4 * n, cudaMemcpyHostToDevice, e->s));
  if (hd.version == 2)  // v^{n-1}, rho^{n-1} of the Verlet scheme, same order
    CUDA_TRY(cudaMemcpyAsync(e->S[0].vrprev, vr + n, 16 * n, cudaMemcpyHostToDevice, e->s));
  CaseDyn d;
  std::memset(&d, 0, sizeof(d));
  d.t = hd.t;
  d.dt = hd.dt;
  d.step = hd.step;
  d.pairs = hd.pairs;
  d.n_out = hd.n_out;
  d.flags = (unsigned)hd.flags;
  d.dtmin_bits = kFloatInfBits;
  CUDA_TRY(cudaMemcpyAsync(e->ddyn, &d, sizeof(d), cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(e->s));
  return SPH_OK;
}

// ---- parity / diagnostics ------------------------------------------------------

int sph_eval_forces(sph_engine e, int32_t icase, float *acc, float *drho, float *mumax,
                    double *dt, int64_t *pairs) {
  int rc = valid_case(e, icase);
  if (rc) return rc;
  const int64_t n = e->slots[icase].n;
  std::vector<CaseDyn> saved(e->cap_cases);
  CUDA_TRY(cudaMemcpyAsync(saved.data(), e->ddyn, sizeof(CaseDyn) * e->cap_cases,
                           cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  std::vector<CaseDyn> fresh = saved;
  for (auto &d : fresh) {
    d.dtmin_bits = kFloatInfBits;
    d.pairs = 0;
  }
  CUDA_TRY(cudaMemcpyAsync(e->ddyn, fresh.data(), sizeof(CaseDyn) * e->cap_cases,
                           cudaMemcpyHostToDevice, e->s));
  enqueue_nl(e);
  const int nl = (int)(e->n_phys - e->n_dead);
  State &Y = e->S[1];
  if (e->mdbc)
    launch_mdbc(e->margin, nl, e->nvalid, e->keysB, Y, e->press, e->cstart, e->nbits, e->dconst,
                e->ddyn, 0, e->s);
  launch_interact(e->margin, e->opt.pi_variant, nl, e->nvalid, e->keysB, Y.posc, Y.velrho,
                  e->press, Y.cid, e->cstart, e->cells_hw, e->nbits, e->dconst, e->ddyn, e->ace,
                  e->mu, 1, e->ext, e->sps ? e->tau4 : nullptr, e->tau2, e->s);
  char *p = e->io;
  float *d_acc = (float *)p;
  p += align256(12 * n);
  float *d_drho = (float *)p;
  p += align256(4 * n);
  float *d_mu = (float *)p;
  launch_scatter_forces(nl, Y.cid, Y.id, icase, 0, e->nvalid, e->ace, e->mu, d_acc, d_drho, d_mu,
                        e->s);
  CUDA_TRY(cudaGetLastError());
  if (acc) CUDA_TRY(cudaMemcpyAsync(acc, d_acc, 12 * n, cudaMemcpyDeviceToHost, e->s));
  if (drho) CUDA_TRY(cudaMemcpyAsync(drho, d_drho, 4 * n, cudaMemcpyDeviceToHost, e->s));
  if (mumax) CUDA_TRY(cudaMemcpyAsync(mumax, d_mu, 4 * n, cudaMemcpyDeviceToHost, e->s));
  CaseDyn d;
  CUDA_TRY(cudaMemcpyAsync(&d, e->ddyn + icase, sizeof(d), cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  CUDA_TRY(cudaMemcpyAsync(e->ddyn, saved.data(), sizeof(CaseDyn) * e->cap_cases,
                           cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  const CaseConst &C = e->hconst[icase];
  if (dt) {
    if (C.dt_fixed > 0)
      *dt = C.dt_fixed;
    else if (d.dtmin_bits >= kFloatInfBits)
      *dt = C.cfl * C.h_d / C.cs0_d;
    else {
      float m;
      std::memcpy(&m, &d.dtmin_bits, 4);
      *dt = C.cfl * (double)m;
    }
  }
  if (pairs) *pairs = (int64_t)d.pairs;
  return SPH_OK;
}

int sph_eval_step(sph_engine e, int32_t icase, int32_t stage, double *pos, float *vel,
                  float *rho, float *acc, float *drho, float *mumax, double *dt,
                  int64_t *pairs) {
  int rc = valid_case(e, icase);
  if (rc) return rc;
  if (stage != 0 && stage != 1) return fail(SPH_ERR_ARG, "stage must be 0 or 1");
  const bool listed = use_list(e);
  if (stage == 1 && (!listed || e->integrator == 1))
    return fail(SPH_ERR_ARG,
                "stage 1 is the half-step evaluation of a Symplectic step over a neighbour "
                "list (pi_variant 3-5); the cell walks (0-2) evaluate it with the stage-0 "
                "kernel on a re-sorted state");
  const int64_t n = e->slots[icase].n;
  const int nl = (int)(e->n_phys - e->n_dead);
  State &Y = e->S[1], &Z = e->S[2];
  cudaStream_t s = e->s;
  const bool reuse = listed && e->opt.pi_variant == 5;
  // the part of the next step that precedes its first evaluation, run for
  // real: the kept list's pending rebuild (which the next step then does not
  // repeat), or the sort of a per-step list or cell walk
  if (reuse) {
    if (!e->s2) CUDA_TRY(cudaStreamCreateWithFlags(&e->s2, cudaStreamNonBlocking));
    if (e->list_stale) launch_need_all(e->cap_cases, e->ddyn, s);
    if (e->list_stale || e->list_dirty)  // a rebuild of every case: ranges may have moved
      CUDA_TRY(cudaMemsetAsync(&e->ctl->rebuild, 1, 2 * sizeof(unsigned int), s));
    e->list_stale = e->list_dirty = false;
    e->cap_err = cudaSuccess;
    enqueue_reuse_rebuild(e, nullptr);
    if (e->cap_err != cudaSuccess) {
      cudaStreamSynchronize(s);
      return fail(SPH_ERR_CUDA, std::string("conditional graph node: ") +
                                    cudaGetErrorString(e->cap_err));
    }
  } else if (listed) {
    enqueue_list_nl(e);
    e->list_stale = true;
  } else {
    enqueue_nl(e);
    if (e->mdbc)
      launch_mdbc(e->margin, nl, e->nvalid, e->keysB, Y, e->press, e->cstart, e->nbits,
                  e->dconst, e->ddyn, 0, s);
  }
  // from here on nothing the next step reads is left changed: the per-case
  // values, the list control and P/rho are restored afterwards
  std::vector<CaseDyn> saved(e->cap_cases), d0(e->cap_cases), d1;
  ListCtl ctl_saved{};
  CUDA_TRY(cudaMemcpyAsync(saved.data(), e->ddyn, sizeof(CaseDyn) * e->cap_cases,
                           cudaMemcpyDeviceToHost, s));
  if (e->ctl)
    CUDA_TRY(cudaMemcpyAsync(&ctl_saved, e->ctl, sizeof(ListCtl), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<CaseDyn> fresh = saved;
  for (auto &d : fresh) {
    d.dtmin_bits = kFloatInfBits;
    d.pairs = d.pairs_fb = d.pairs_bf = 0;
    d.flags = 0;
  }
  CUDA_TRY(cudaMemcpyAsync(e->ddyn, fresh.data(), sizeof(CaseDyn) * e->cap_cases,
                           cudaMemcpyHostToDevice, s));
  float *press_saved = (float *)e->keysD;  // unused by the list steps' launches
  if (nl > 0)
    CUDA_TRY(cudaMemcpyAsync(press_saved, e->press, 4 * (size_t)nl, cudaMemcpyDeviceToDevice, s));
  if (listed)
    enqueue_list_first(e, nullptr, e->mu);
  else
    launch_interact(e->margin, e->opt.pi_variant, nl, e->nvalid, e->keysB, Y.posc, Y.velrho,
                    e->press, Y.cid, e->cstart, e->cells_hw, e->nbits, e->dconst, e->ddyn,
                    e->ace, e->mu, 1, e->ext, e->sps ? e->tau4 : nullptr, e->tau2, s);
  CUDA_TRY(cudaMemcpyAsync(d0.data(), e->ddyn, sizeof(CaseDyn) * e->cap_cases,
                           cudaMemcpyDeviceToHost, s));
  if (stage == 1) {
    d1.resize(e->cap_cases);
    enqueue_list_half(e, nullptr, e->mu);
    CUDA_TRY(cudaMemcpyAsync(d1.data(), e->ddyn, sizeof(CaseDyn) * e->cap_cases,
                             cudaMemcpyDeviceToHost, s));
  }
  // results and the evaluated state, in the caller's order
  const uint32_t *keys = stage == 1 ? e->keysC : e->keysB;
  const State st = stage == 1 ? half_state(Y, Z) : Y;
  char *p = e->io;
  double *d_pos = (double *)p;
  p += align256(24 * n);
  float *d_vel = (float *)p;
  p += align256(12 * n);
  float *d_rho = (float *)p;
  p += align256(4 * n);
  float *d_acc = (float *)p;
  p += align256(12 * n);
  float *d_drho = (float *)p;
  p += align256(4 * n);
  float *d_mu = (float *)p;
  launch_scatter_forces(nl, Y.cid, Y.id, icase, 0, e->nvalid, e->ace, e->mu, d_acc, d_drho, d_mu,
                        s, keys, e->nbits);
  launch_export((int)e->n_phys, keys, st, e->dconst, icase, 0, e->nbits, d_pos, d_vel, d_rho,
                nullptr, s);
  CUDA_TRY(cudaGetLastError());
  if (pos) CUDA_TRY(cudaMemcpyAsync(pos, d_pos, 24 * n, cudaMemcpyDeviceToHost, s));
  if (vel) CUDA_TRY(cudaMemcpyAsync(vel, d_vel, 12 * n, cudaMemcpyDeviceToHost, s));
  if (rho) CUDA_TRY(cudaMemcpyAsync(rho, d_rho, 4 * n, cudaMemcpyDeviceToHost, s));
  if (acc) CUDA_TRY(cudaMemcpyAsync(acc, d_acc, 12 * n, cudaMemcpyDeviceToHost, s));
  if (drho) CUDA_TRY(cudaMemcpyAsync(drho, d_drho, 4 * n, cudaMemcpyDeviceToHost, s));
  if (mumax) CUDA_TRY(cudaMemcpyAsync(mumax, d_mu, 4 * n, cudaMemcpyDeviceToHost, s));
  // restore
  if (nl > 0)
    CUDA_TRY(cudaMemcpyAsync(e->press, press_saved, 4 * (size_t)nl, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(e->ddyn, saved.data(), sizeof(CaseDyn) * e->cap_cases,
                           cudaMemcpyHostToDevice, s));
  if (e->ctl)
    CUDA_TRY(cudaMemcpyAsync(e->ctl, &ctl_saved, sizeof(ListCtl), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const std::vector<CaseDyn> &dl = stage == 1 ? d1 : d0;
  const unsigned bad = dl[icase].flags;
  if (bad & kFlagNaN) return fail(SPH_ERR_UNSTABLE, "NaN/Inf in the interaction");
  if (bad & kFlagListFull)
    return fail(SPH_ERR_STATE, "a particle has more neighbour-list candidates than the list holds");
  if (bad & kFlagSkin)
    return fail(SPH_ERR_UNSTABLE, "the half step left the neighbour list's skin");
  const CaseConst &C = e->hconst[icase];
  if (dt) {
    const unsigned bits = d0[icase].dtmin_bits;
    if (C.dt_fixed > 0)
      *dt = C.dt_fixed;
    else if (bits >= kFloatInfBits)
      *dt = C.cfl * C.h_d / C.cs0_d;
    else {
      float m;
      std::memcpy(&m, &bits, 4);
      *dt = C.cfl * (double)m;
    }
  }
  if (pairs)
    *pairs = (int64_t)(stage == 1 ? d1[icase].pairs - d0[icase].pairs : d0[icase].pairs);
  return SPH_OK;
}

int sph_eval_sps(sph_engine e, int32_t icase, float *tau6) {
  int rc = valid_case(e, icase);
  if (rc) return rc;
  if (!tau6) return fail(SPH_ERR_ARG, "null output");
  if (!e->tau4) return fail(SPH_ERR_STATE, "no case of this engine uses visc_mode 1");
  const int64_t n = e->slots[icase].n;
  enqueue_nl(e);
  const int nl = (int)(e->n_phys - e->n_dead);
  State &Y = e->S[1];
  launch_strain(e->margin, nl, e->nvalid, e->keysB, Y.posc, Y.velrho, Y.cid, e->cstart,
                e->cells_hw, e->nbits, e->dconst, e->tau4, e->tau2, e->s);
  float *d_tau = (float *)e->io;  // 24 n bytes <= io_bytes (48 per particle)
  CUDA_TRY(cudaMemsetAsync(d_tau, 0, 24 * n, e->s));
  launch_scatter_tau(nl, Y.cid, Y.id, icase, e->nvalid, e->tau4, e->tau2, d_tau, e->s);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(tau6, d_tau, 24 * n, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  return SPH_OK;
}

int sph_eval_boundary(sph_engine e, int32_t icase, float *vel, float *rho) {
  int rc = valid_case(e, icase);
  if (rc) return rc;
  if (!e->mdbc) return fail(SPH_ERR_STATE, "no case of this engine uses boundary_mode 1");
  const int64_t n = e->slots[icase].n;
  enqueue_nl(e);
  const int nl = (int)(e->n_phys - e->n_dead);
  State &Y = e->S[1];
  launch_mdbc(e->margin, nl, e->nvalid, e->keysB, Y, e->press, e->cstart, e->nbits, e->dconst,
              e->ddyn, 0, e->s);
  char *p = e->io;
  float *d_vel = (float *)p;
  p += align256(12 * n);
  float *d_rho = (float *)p;
  launch_export(nl, e->keysB, Y, e->dconst, icase, 0, e->nbits, nullptr, vel ? d_vel : nullptr,
                rho ? d_rho : nullptr, nullptr, e->s);
  CUDA_TRY(cudaGetLastError());
  if (vel) CUDA_TRY(cudaMemcpyAsync(vel, d_vel, 12 * n, cudaMemcpyDeviceToHost, e->s));
  if (rho) CUDA_TRY(cudaMemcpyAsync(rho, d_rho, 4 * n, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  return SPH_OK;
}

int sph_get_order(sph_engine e, int32_t icase, int64_t *ids, int64_t *cells, int64_t *n_inside) {
  int rc = valid_case(e, icase);
  if (rc) return rc;
  enqueue_nl(e);
  const int64_t np = e->n_phys;
  std::vector<uint32_t> keys(np), id(np);
  std::vector<uint16_t> cid(np);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(keys.data(), e->keysB, 4 * np, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaMemcpyAsync(id.data(), e->S[1].id, 4 * np, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaMemcpyAsync(cid.data(), e->S[1].cid, 2 * np, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  const uint32_t kout = key_out(e->nbits), kdead = key_dead(e->nbits);
  const uint32_t cb = e->slots[icase].cellbase;
  int64_t j = 0, inside = 0;
  for (int64_t i = 0; i < np - e->n_dead; i++) {
    if (cid[i] != icase || keys[i] == kdead) continue;
    if (ids) ids[j] = id[i];
    if (cells) cells[j] = keys[i] >= kout ? -1 : (int64_t)(key_cell(keys[i], e->nbits) - cb);
    inside += keys[i] < kout;
    j++;
  }
  if (n_inside) *n_inside = inside;
  return SPH_OK;
}

int sph_pair_stats(sph_engine e, int32_t icase, int64_t *count, uint64_t *hash) {
  int rc = valid_case(e, icase);
  if (rc) return rc;
  const int64_t n = e->slots[icase].n;
  enqueue_nl(e);
  char *p = e->io;
  long long *d_count = (long long *)p;
  p += align256(8 * n);
  unsigned long long *d_hash = (unsigned long long *)p;
  CUDA_TRY(cudaMemsetAsync(d_count, 0, 8 * n, e->s));
  CUDA_TRY(cudaMemsetAsync(d_hash, 0, 8 * n, e->s));
  launch_pair_stats((int)(e->n_phys - e->n_dead), e->nvalid, e->keysB, e->S[1], e->cstart,
                    e->cells_hw, e->nbits, e->dconst, icase, 0, d_count, d_hash, e->s);
  CUDA_TRY(cudaGetLastError());
  if (count) CUDA_TRY(cudaMemcpyAsync(count, d_count, 8 * n, cudaMemcpyDeviceToHost, e->s));
  if (hash) CUDA_TRY(cudaMemcpyAsync(hash, d_hash, 8 * n, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  return SPH_OK;
}

// ---- serving pool --------------------------------------------------------------

int sph_pool_create(int64_t max_particles, int64_t max_cells, int32_t max_cases, void *stream,
                    sph_alloc_fn alloc, sph_free_fn free_fn, void *alloc_ctx, sph_engine *out) {
  if (!out) return fail(SPH_ERR_ARG, "null output handle");
  *out = nullptr;
  if (max_particles <= 0 || max_particles > (int64_t(1) << 31) - 1 || max_cells <= 0 ||
      max_cells > (int64_t(1) << 30) || max_cases <= 0 || max_cases > 65535)
    return fail(SPH_ERR_ARG, "bad pool capacity");
  sph_engine e = new sph_engine_t();
  int rc = init_engine(e, stream, alloc, free_fn, alloc_ctx);
  if (rc) {
    delete e;
    return rc;
  }
  e->pool = true;
  e->cap_p = max_particles;
  e->cap_cells = max_cells;
  e->cap_cases = max_cases;
  e->nbits = bits_for(max_cells);
  e->slots.resize(max_cases);
  e->hconst.resize(max_cases);
  e->free_cells.push_back({0, max_cells});
  // per-step list for the pool's cases, sized for h up to 1.2 sqrt(3) dp and any
  // cell size; a case needing more records turns the list off (admission)
  e->list_ok = max_particles < kListMaxParticles;
  if (e->list_ok) {
    const double hq = 1.2 * std::sqrt(3.0);
    for (int cm = 0; cm < 3; cm++) e->list_cap = std::max(e->list_cap, list_records_needed(cm, hq, 1.0));
    e->list_default = 5;  // the list kept across steps (4: cases equal alone, bit for bit)
    e->opt.pi_variant = 5;
  }
  rc = allocate(e);
  if (rc == SPH_OK) {
    cudaError_t err = cudaStreamSynchronize(e->s);
    if (err != cudaSuccess) rc = fail(SPH_ERR_CUDA, cudaGetErrorString(err));
  }
  if (rc) {
    e->release_all();
    delete e;
    return rc;
  }
  *out = e;
  return SPH_OK;
}

int sph_pool_admit(sph_engine e, const sph_case_params *params, const sph_particles *parts,
                   double t_end, int32_t *slot) {
  if (!e || !e->pool) return fail(SPH_ERR_STATE, "not a pool engine");
  if (!slot) return fail(SPH_ERR_ARG, "null slot pointer");
  int rc = check_particles(params, parts);
  if (rc) return rc;
  Grid g;
  rc = make_grid(*params, g);
  if (rc) return rc;
  int used = 0;
  for (auto &s : e->slots) used += s.used;
  if (params->integrator != 0)
    return fail(SPH_ERR_ARG, "pools run the Symplectic scheme (integrator 0)");
  // (the pool's tau buffers exist from creation; the flags only grow)
  const bool sym0 = sym_on(e);
  e->ext = e->ext || params->ddt_mode == 2 || params->visc_mode == 1;
  e->sps = e->sps || params->visc_mode == 1;
  e->mdbc = e->mdbc || params->boundary_mode == 1;
  if (e->list_ok && list_records_needed(params->cell_mode, params->h, params->dp) > e->list_cap)
    e->list_ok = false;  // from now on the pool runs two neighbour lists per step
  e->opt.pi_variant = resolve_variant(e, e->opt.pi_variant);
  // the half lists of the pair-once walk no longer serve: every case rebuilds
  if (sym0 && !sym_on(e)) e->list_stale = true;
  if (used == 0) e->margin = g.margin;
  if (g.margin != e->margin) return fail(SPH_ERR_ARG, "cell_mode differs from the pool's cases");
  int free_slot = -1;
  for (int c = 0; c < e->cap_cases; c++)
    if (!e->slots[c].used) {
      free_slot = c;
      break;
    }
  if (free_slot < 0) return fail(SPH_ERR_BUSY, "no free case slot");
  if (e->n_phys + parts->n > e->cap_p) return fail(SPH_ERR_BUSY, "not enough particle memory");
  int fr = -1;
  for (size_t r = 0; r < e->free_cells.size(); r++)
    if (e->free_cells[r].second - e->free_cells[r].first >= g.ncells) {
      fr = (int)r;
      break;
    }
  if (fr < 0) return fail(SPH_ERR_BUSY, "not enough cell-table memory");
  const int64_t cb = e->free_cells[fr].first;
  e->free_cells[fr].first += g.ncells;
  if (e->free_cells[fr].first == e->free_cells[fr].second)
    e->free_cells.erase(e->free_cells.begin() + fr);
  rc = set_slot(e, free_slot, params, parts, g, (uint32_t)cb, t_end);
  if (rc == SPH_OK) rc = upload_case(e, free_slot, parts, e->n_phys);
  if (rc) return rc;
  e->n_phys += parts->n;
  e->cells_hw = std::max<int64_t>(e->cells_hw, cb + g.ncells);
  e->drop_graphs();
  *slot = free_slot;
  return SPH_OK;
}

int sph_pool_step(sph_engine e, int64_t nsteps, int32_t *finished, int32_t *n_finished) {
  if (!e || !e->pool) return fail(SPH_ERR_STATE, "not a pool engine");
  int rc = sph_step(e, nsteps);
  if (rc) return rc;
  std::vector<CaseDyn> d(e->cap_cases);
  CUDA_TRY(cudaMemcpyAsync(d.data(), e->ddyn, sizeof(CaseDyn) * e->cap_cases,
                           cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  int k = 0;
  for (int c = 0; c < e->cap_cases; c++)
    if (e->slots[c].used && e->slots[c].t_end > 0 && d[c].t >= e->slots[c].t_end) {
      if (finished) finished[k] = c;
      k++;
    }
  if (n_finished) *n_finished = k;
  return SPH_OK;
}

int sph_pool_release(sph_engine e, int32_t slot) {
  if (!e || !e->pool) return fail(SPH_ERR_STATE, "not a pool engine");
  int rc = valid_case(e, slot);
  if (rc) return rc;
  launch_release((int)e->n_phys, e->S[0].cid, slot, e->nbits, e->keysA, e->s);
  e->hconst[slot].active = 0;
  CUDA_TRY(cudaMemcpyAsync(e->dconst + slot, &e->hconst[slot], sizeof(CaseConst),
                           cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(e->s));
  Slot &S = e->slots[slot];
  e->n_dead += S.n;
  // return the cell range (merge neighbours)
  e->free_cells.push_back({S.cellbase, S.cellbase + S.ncells});
  std::sort(e->free_cells.begin(), e->free_cells.end());
  std::vector<std::pair<int64_t, int64_t>> merged;
  for (auto &r : e->free_cells) {
    if (!merged.empty() && merged.back().second == r.first)
      merged.back().second = r.second;
    else
      merged.push_back(r);
  }
  e->free_cells.swap(merged);
  S = Slot();
  e->cells_hw = 0;
  for (auto &s : e->slots)
    if (s.used) e->cells_hw = std::max<int64_t>(e->cells_hw, (int64_t)s.cellbase + s.ncells);
  e->drop_graphs();
  e->list_dirty = true;  // the other cases' indices move: their lists are re-expressed
  return SPH_OK;
}

int sph_pool_usage(sph_engine e, int64_t *particles_used, int64_t *cells_used,
                   int32_t *cases_used) {
  if (!e) return fail(SPH_ERR_ARG, "null engine");
  int64_t cells = 0;
  int cases = 0;
  for (auto &s : e->slots)
    if (s.used) {
      cells += s.ncells;
      cases++;
    }
  if (particles_used) *particles_used = e->n_phys - e->n_dead;
  if (cells_used) *cells_used = cells;
  if (cases_used) *cases_used = cases;
  return SPH_OK;
}

void sph_destroy(sph_engine e) {
  if (!e) return;
  e->release_all();
  delete e;
}

}  // extern "C"
