// sph_kernels.cuh -- host launchers of the kernels in sph_kernels.cu.
#pragma once
#include "sph_internal.cuh"

namespace sph {

void launch_upload(int n, const double *pos, const float *vel, const float *rho,
                   const uint8_t *type, const int32_t *group, int slot, uint32_t id_base,
                   const CaseConst *cc, CaseDyn *dyn, int nbits, State st, uint32_t *keys,
                   int dst0, const float *ghost, cudaStream_t s);
// ref_src / ref_dst (or null): also gather the kept list's build positions.
void launch_reorder(int n, const uint32_t *perm, const uint32_t *keys_sorted,
                    const float4 *posc, const float4 *velrho, const uint32_t *id,
                    const uint16_t *cid, const uint8_t *code, const float4 *vrprev,
                    const float4 *ghost, State dst, float *press, const CaseConst *cc,
                    CaseDyn *dyn, int nbits, cudaStream_t s, const float4 *ref_src = nullptr,
                    float4 *ref_dst = nullptr);
// Words of temporary storage launch_cells needs for cap_cells cells.
size_t cells_temp_words(int64_t cap_cells);
// Cell start table of the sorted keys (and nvalid); returns kernels launched.
int launch_cells(int n, const uint32_t *keys, uint32_t *cstart, int64_t cap_cells, int nbits,
                 int *nvalid, uint32_t *tmp, cudaStream_t s);
// Strain pass of the laminar + SPS model alone (tau/rho of Eq 25, sorted order).
void launch_strain(int margin, int n, const int *nvalid, const uint32_t *keys,
                   const float4 *posc, const float4 *velrho, const uint16_t *cid,
                   const uint32_t *cstart, int64_t cap_cells, int nbits, const CaseConst *cc,
                   float4 *tau4, float2 *tau2, cudaStream_t s);
void launch_scatter_tau(int n, const uint16_t *cid, const uint32_t *id, int slot,
                        const int *nvalid, const float4 *tau4, const float2 *tau2, float *out,
                        cudaStream_t s);
void launch_interact(int margin, int variant, int n, const int *nvalid, const uint32_t *keys,
                     const float4 *posc, const float4 *velrho, const float *press,
                     const uint16_t *cid, const uint32_t *cstart, int64_t cap_cells, int nbits,
                     const CaseConst *cc, CaseDyn *dyn, float4 *ace, float *mu, int want_dt,
                     bool ext, float4 *tau4, float2 *tau2, cudaStream_t s);
void launch_dt(int ncases, const CaseConst *cc, CaseDyn *dyn, cudaStream_t s);
void launch_end_step(int ncases, const CaseConst *cc, CaseDyn *dyn, cudaStream_t s);
void launch_predictor(int n, const uint32_t *keys_in, State src, const float4 *ace,
                      const CaseConst *cc, CaseDyn *dyn, int nbits, float4 *posc_out,
                      float4 *velrho_out, uint32_t *keys_out, cudaStream_t s);
// mDBC boundary values (Eq 38-39) on the sorted state st, before an
// interaction; stage 0: wall velocity at t, 1: at t + dt/2.  list: st is in
// the cells of a neighbour list's build (offsets up to skin/2 outside them).
void launch_mdbc(int margin, int n, const int *nvalid, const uint32_t *keys, State st,
                 float *press, const uint32_t *cstart, int nbits, const CaseConst *cc,
                 const CaseDyn *dyn, int stage, cudaStream_t s, bool list = false);
// Neighbour list (Symplectic scheme, boundary_mode 0): build on state n
// with radius 2h + skin; interaction over the list; predictor and corrector
// that keep the order and the cells of the build.
// Per-case skin and build mode of the next build (fresh_all: every case
// builds from its state; else only the cases that need it, after the cell
// table of the sort); clears the rebuild request and counts the build.
void launch_list_begin(int ncases, const CaseConst *cc, CaseDyn *dyn, ListCtl *ctl,
                       float extra, int fresh_all, const uint32_t *cstart, int64_t cap_cells,
                       cudaStream_t s);
// Kept list, before a rebuild's sort: the cases that need no rebuild enter
// the sort with their build keys and build-cell state.
void launch_select(int n, const uint16_t *cid, const CaseConst *cc, const CaseDyn *dyn,
                   const uint32_t *keys_build, const float4 *posc_build, uint32_t *keys,
                   float4 *posc, const ListCtl *ctl, cudaStream_t s);
// The sort, reorder and scatter of a kept-list rebuild: the particles of the
// cases that need a list (every particle when ctl->full), sorted by key within
// the slots they occupy, from src (x) into dst (y) and keys_dst, with P/rho,
// the max |v|^2 per case and the build positions (ref_src -> ref_dst).
// Scratch: tmp (rb_temp_words(n) words), idx, kc, kc_sorted, perm ([n] each)
// and sort_tmp (radix_sort_temp_bytes(n)).
size_t rb_temp_words(int64_t n);
void launch_rebuild_sort(int n, const ListCtl *ctl, const uint32_t *keys, State src, State dst,
                         uint32_t *keys_dst, float *press, const CaseConst *cc, CaseDyn *dyn,
                         int nbits, const float4 *ref_src, float4 *ref_dst, uint32_t *tmp,
                         uint32_t *idx, uint32_t *kc, uint32_t *kc_sorted, uint32_t *perm,
                         void *sort_tmp, cudaStream_t s);
// Marks every case's kept list for a rebuild.
void launch_need_all(int ncases, CaseDyn *dyn, cudaStream_t s);
// The list alone (the candidate test of the compacted loop, no pair terms);
// ref (or null) receives every target's position at the build, and then the
// cases' build modes apply (ref_src: the previous build positions, gathered).
void launch_build_list(int margin, int n, const int *nvalid, const uint32_t *keys,
                       const float4 *posc, const float4 *velrho, const float *press,
                       const uint16_t *cid, const uint32_t *cstart, int64_t cap_cells, int nbits,
                       const CaseConst *cc, CaseDyn *dyn, float4 *ace, uint2 *list, int cap,
                       uint16_t *count, float4 *ref, const float4 *ref_src, cudaStream_t s,
                       bool half = false, bool wide = false);
// First evaluation of the list step: the compacted pair loop on state n that
// also writes every target's list (chunk records, radius 2h + skin) and count.
void launch_interact_build(int margin, int n, const int *nvalid, const uint32_t *keys,
                           const float4 *posc, const float4 *velrho, const float *press,
                           const uint16_t *cid, const uint32_t *cstart, int64_t cap_cells,
                           int nbits, const CaseConst *cc, CaseDyn *dyn, float4 *ace,
                           uint2 *list, int cap, uint16_t *count, bool ext, float4 *tau4,
                           float2 *tau2, cudaStream_t s, float *mu = nullptr);
void launch_interact_list(int n, const int *nvalid, const uint32_t *keys, const float4 *posc,
                          const float4 *velrho, const float *press, const uint16_t *cid,
                          const uint32_t *cstart, int64_t cap_cells, int nbits,
                          const CaseConst *cc, CaseDyn *dyn, float4 *ace, int want_dt,
                          const uint2 *list, int cap, const uint16_t *count, bool ext,
                          float4 *tau4, float2 *tau2, cudaStream_t s, float *mu = nullptr,
                          int block = 128, int lanes = 1, float4 *sym_sum = nullptr,
                          unsigned *sym_mu = nullptr, const uint32_t *wide_keys = nullptr);
void launch_predictor_list(int n, const uint32_t *keys_in, State src, const float4 *ace,
                           const CaseConst *cc, CaseDyn *dyn, int nbits, float4 *posc_out,
                           float4 *velrho_out, uint32_t *keys_out, float *press,
                           const float4 *ref, cudaStream_t s);
// Corrector of the list kept across steps: state n+1 to x (normalised, keys)
// and in place to y (the build's cells, P/rho to press); requests a rebuild
// through ctl when the next step could leave the skin.
void launch_corrector_reuse(int n, const uint32_t *keys_n, const uint32_t *keys_half, State y,
                            const float4 *velrho_half, const float4 *ace, const float4 *ref,
                            const CaseConst *cc, CaseDyn *dyn, int nbits, State x,
                            uint32_t *keys_next, float *press, ListCtl *ctl, cudaStream_t s);
// One-thread kernel: sets conditional handle h to ctl->rebuild != 0.
void launch_decide(cudaGraphConditionalHandle h, const ListCtl *ctl, cudaStream_t s);
// Brute-force check of the list against the evaluated state (tests).
void launch_list_check(int n, const int *nvalid, const uint32_t *keys, const float4 *posc,
                       const uint16_t *cid, const CaseConst *cc, int nbits, const uint2 *list,
                       int cap, const uint16_t *count, ListCtl *ctl, cudaStream_t s,
                       bool half = false, const uint32_t *wide_keys = nullptr);
void launch_corrector_list(int n, const uint32_t *keys_n, const uint32_t *keys_half, State sn,
                           const float4 *velrho_half, const float4 *ace, const CaseConst *cc,
                           CaseDyn *dyn, int nbits, State x, uint32_t *keys_next,
                           cudaStream_t s);
// Verlet step (Eq 30-31) from the sorted state src to dst (same order).
void launch_verlet(int n, const uint32_t *keys_in, State src, const float4 *ace,
                   const CaseConst *cc, CaseDyn *dyn, int nbits, State dst, uint32_t *keys_out,
                   cudaStream_t s);
// The same with the list kept across steps: state n+1 also in place into y
// (the build's cells, P/rho to press); rebuild requested through ctl.
void launch_verlet_reuse(int n, const uint32_t *keys_in, State y, const float4 *ace,
                         const CaseConst *cc, CaseDyn *dyn, int nbits, State x,
                         uint32_t *keys_out, const float4 *ref, float *press, ListCtl *ctl,
                         cudaStream_t s);
void launch_corrector(int n, const uint32_t *perm2, const uint32_t *keys_half,
                      const uint32_t *keys_n, State sn, State x, const float4 *ace,
                      const CaseConst *cc, CaseDyn *dyn, int nbits, uint32_t *keys_next,
                      cudaStream_t s);
void launch_export(int n, const uint32_t *keys, State st, const CaseConst *cc, int slot,
                   uint32_t id_base, int nbits, double *pos, float *vel, float *rho,
                   float *press, cudaStream_t s);
void launch_import_raw(int n, const int32_t *cell, const float4 *posc, const float4 *velrho,
                       const uint8_t *type, const int32_t *group, int slot, uint32_t id_base,
                       const CaseConst *cc, int nbits, State st, uint32_t *keys, int dst0,
                       const float *ghost, cudaStream_t s);
void launch_scatter_forces(int n, const uint16_t *cid, const uint32_t *id, int slot,
                           uint32_t id_base, const int *nvalid, const float4 *ace,
                           const float *mu, float *acc_out, float *drho_out, float *mu_out,
                           cudaStream_t s, const uint32_t *keys = nullptr, int nbits = 0);
void launch_pair_stats(int n, const int *nvalid, const uint32_t *keys, State st,
                       const uint32_t *cstart, int64_t cap_cells, int nbits, const CaseConst *cc,
                       int slot, uint32_t id_base, long long *count, unsigned long long *hash,
                       cudaStream_t s);
void launch_diag(int n, const uint32_t *keys, State st, const CaseConst *cc, int slot,
                 int nbits, double *part, int nparts, double *out, cudaStream_t s);
void launch_release(int n, const uint16_t *cid, int slot, int nbits, uint32_t *keys,
                    cudaStream_t s);

}  // namespace sph
