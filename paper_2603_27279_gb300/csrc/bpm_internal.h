// Internal declarations of the GB300 bonded-particle rod library.
//
// Device data layout (all owned by the handle, one cudaMalloc arena):
//   state, SoA:  x[3][N], q[4][N], v[3][N], w[3][N]      (float64)
//   forces, SoA: f[3][N], t[3][N]                         (float64)
//   dipoles:     m[3][N] (space frame, FP64); for the mixed path also
//                xh[3][N], xl[3][N] (FP32 hi/lo split of x) and mf[3][N];
//                for the float-float path xq[9][N] (fixed-binade digits of
//                x) and mq[6][N] (hi and lo parts of m)
//   per particle constants: m_body[3][N], mass[N], inertia[N], 1/mass[N],
//                1/inertia[N],
//                flags[N] (bit 0 clamped, bit 1 "bond to particle k+1"),
//                rod_of[N]
//   per bond slot k (bond k -> k+1 when flags[k] & 2), SoA [8][N]:
//                rest direction r^_i (3), rest length L, K_r, K_s, K_t, K_b
//   bond damping (optional): g per rod [4][R], measures [2][3][N], parity
//   contact (optional): cell list (key, bucket counts / starts, order) and
//                tangential histories [2][cap][N] (partner, xi, counts)
//   dipole partial sums, SoA [S][7][N]: F~ (3), H~ (3), sum b/r^5 (1)
//   energy scratch [5][N]
// SoA keeps every per-particle load of a warp coalesced; the j-tiles of the
// dipole kernels are staged through shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bpm.h"

namespace bpm {

enum : uint8_t { F_CLAMPED = 1, F_BOND_RIGHT = 2 };

// Uniform and time-dependent parts of the external field, by value.
struct Field {
    double B[3];
    double rot_amp, rot_omega;
    double e1[3], e2[3];
    double G[9];
    double x0[3];
    int has_grad;
    const double* B_rod;  // device [3][R] SoA or nullptr
    int64_t n_rods;
};

// Device view of a system, passed by value to every kernel.
struct Sys {
    int64_t n;
    double *x, *q, *v, *w;    // SoA state
    double *f, *t;            // SoA force / torque
    double* m;                // SoA space-frame dipoles
    float *xh, *xl, *mf;      // mixed-precision copies (may be null)
    float *xq, *mq;           // float-float copies (BPM_FF, may be null):
                              // position digits [3 digits][3][N], moment hi/lo [2][3][N]
    int q_exp;                // BPM_FF: the finest position digit is 2^q_exp
    const double* m_body;     // SoA body-frame dipoles
    const double* mass;
    const double* inertia;    // 2/5 m R^2
    const double* inv_mass;   // 1/m
    const double* inv_inertia;
    const uint8_t* flags;
    const int32_t* rod_of;
    const double* bond;       // SoA [8][N]
    double* tdev;             // simulation time (device scalar)
    int* err;                 // first failing step + 1 (0 = ok)
    int* step_counter;        // device step index for error reports
    int count_step;           // 1: the bond kernel advances step_counter
    double damping, dt, c;
    Field field;
    // dipole partials
    double* part;             // [S][7][N]
    const uint8_t* nslot;     // per particle: number of valid slots
    int S;
    int slots_reduced;        // 1: k_reduce_slots has summed the slots into slot 0
    // energy scratch
    double* e_part;           // [5][N]
    // bond-level damping (null when the system has none)
    const double* bond_g;     // per rod SoA [4][R]: g_r, g_s, g_t, g_b
    double* hist;             // two levels [2][3][N] of (gamma, psi, theta) per bond slot; NaN = none
    int* hist_gen;            // level parity (bond measures and contact histories):
                              // current = level (gen & 1), previous = the other
    int* ct_valid;            // contact: [2] 1 when a level holds a record (null: no contact)
};

// Contact between non-bonded particles: parameters, the per-step cell list
// (spatial hash of cells of side `cell`, H buckets) and the two levels of
// tangential histories, SoA [level][slot][N].
struct Contact {
    double E_star, G_star, mu, gamma_n, gamma_t;
    double inv_cell;          // 1 / cell side (cell side = largest contact distance)
    int exclude, cap;
    uint32_t H;               // buckets, a power of two
    int* key;                 // [N] bucket of each particle
    int* count;               // [H] particles per bucket (zero between builds)
    int* start;               // [H+1] exclusive prefix sums
    int* order;               // [N] particles grouped by bucket, ascending within one
    int* block_sums;          // scan scratch
    int* partner;             // [2][cap][N]
    double* xi;               // [2][3][cap][N]
    int* ncont;               // [2][N]
    int* overflow;            // set when a particle has more than cap contacts
    const double* radius;     // [N] particle radii
    float* xf;                // [3][N] FP32 copies of x for the candidate filter
    const float* radf;        // [N] FP32 radii
};

// Lattice Boltzmann fluid and its penalty coupling (lattice units).
struct Lbm {
    int nx, ny, nz, n_sub;
    double tau;
    double omega, gfac;       // 1 / tau and 1 - 1 / (2 tau)
    double body[3];           // uniform force density on the fluid
    float omegaf, gfacf, bodyf[3];  // the same in FP32 (FP32 storage)
    float omega2[2], gfac2[2], body2[3][2];  // the same as float-float (hi, lo) pairs
    void* f[2];               // [19][nodes] post-collision distributions: FP64, or FP32 deviations f - w
    void* F;                  // [3][nodes] particle reaction for the next LBM step (storage type)
    double* U;                // [3][N] fluid velocity interpolated at the particles
    const uint8_t* coupled;   // [N] 1 = coupled, or null (all)
    int fp32;                 // 1: FP32 storage and collision
    int ff;                   // 1: FP64 storage, float-float collision (BPM_FF handles)
};

// Dipole work item: i in [i0, i0+ni), j in [j0, j0+nj), written to slot.
struct WorkItem {
    int32_t i0, ni, j0, nj, slot, pad0, pad1, pad2;
};

// Device buffers of the adjoint sweep (SoA [c][N] each).
struct AdjBuf {
    double *ax, *aq, *av, *aw;  // adjoints of the state P_k (x, q, vh, wh)
    double *aF, *aT;            // adjoints of the forces at the current snapshot
    double *amb, *aB;           // d/d(body dipoles) and per-particle pieces of d/dB
    double *m, *mu, *dx, *dm;   // scratch: m, lambda_tau x m
    double *bL, *bR;            // bond VJP pieces [7][N] for particles k and k+1
    double* dpart;              // dipole VJP pieces [S][6][N] (d/dx, d/dm per j-chunk or partner tile)
    int S;                      // j-chunks (or 32-particle tiles, symmetric form) of the dipole VJP
    int sym;                    // symmetric dipole VJP (one warp per pair of tiles)
    float* ffbuf;               // BPM_FF handles: float-float VJP inputs [adj_ff_comp()][N], else null
};

// ---------------------------------------------------------------------------
// kernel launchers (each defined in its own translation unit)
// ---------------------------------------------------------------------------
// bond + Zeeman + damping + dipole orientation (+ bond/Zeeman energies)
// m_given: the dipole moments m were written by launch_orient and are read,
// not computed (the form that runs beside the dipole kernel; no energy);
// grid > 0: at most that many blocks, looping over the particle groups
cudaError_t launch_bond(const Sys& s, bool energy, bool mixed_copies, bool m_given, int grid, cudaStream_t st);
// m = q m~ q* for every particle, and the FP32 copies of x and m when asked
cudaError_t launch_orient(const Sys& s, bool mixed_copies, cudaStream_t st);

// dipole all-pairs partial sums over a work list
struct DipoleCfg {
    int threads;     // threads per block
    int ipt;         // i particles per thread (mixed path)
    int blocks;      // persistent grid size
    int sym;         // 1: symmetric kernel over supertile pairs
    int g;           // tiles per supertile (symmetric kernel)
};
// beside: the form that runs beside the bond kernel (the FP32-pair kernel
// with its registers capped so that both kernels' blocks fit an SM)
cudaError_t launch_dipole(const Sys& s, bool mixed, const WorkItem* items, int n_items,
                          int* counter, const DipoleCfg& cfg, cudaStream_t st, bool beside = false);
int dipole_tile_i(bool mixed, const DipoleCfg& cfg);  // i particles per item
// symmetric kernel (each unordered pair once): items are supertile pairs
// (pad0 = j-side slot, pad1 = 1 on the diagonal)
int dipole_sym_tile(bool mixed);
// symmetric kernels with warp tiles and one warp per pair of tiles (plan
// param 0; 32-particle tiles in FP64 and float-float, 64 in FP32 pairs):
// items are tile pairs (pad0 = j-side slot, pad1 = 1 on the diagonal)
int dipole_symw_blocks_per_sm();
int dipole_symw_ff_blocks_per_sm();
int dipole_symw_mixed_blocks_per_sm();
cudaError_t launch_dipole_symw_mixed(const Sys& s, const WorkItem* items, int n_items, int* counter, int blocks,
                                     cudaStream_t st);
cudaError_t launch_dipole_symw_fp64(const Sys& s, const WorkItem* items, int n_items, int* counter, int blocks,
                                    cudaStream_t st);
cudaError_t launch_dipole_symw_ff(const Sys& s, const WorkItem* items, int n_items, int* counter, int blocks,
                                  cudaStream_t st);
int dipole_sym_blocks_per_sm(bool mixed, int g);
// What one block of a kernel holds on an SM: registers per thread as
// allocated (multiples of 8), threads, and shared memory (static and
// dynamic), for sizing two kernels that run side by side.
struct BlockRes {
    int regs = 0, threads = 0, smem = 0;
};
BlockRes block_res_of(const void* fn, int threads, int dyn_smem);
// the dipole kernel of a plan (sym false: ordered; g = 0: warp tiles), and
// the bond kernel's form beside it (m given)
BlockRes dipole_block_res(bool mixed, bool sym, int g, bool beside = false);
BlockRes dipole_ff_block_res(int g);
BlockRes bond_side_block_res(bool damp);
// ragged: some item's particle ranges end inside a tile (the FP64 kernel then
// skips padding warps and subtiles; the mixed kernel ignores it)
cudaError_t launch_dipole_sym(const Sys& s, bool mixed, const WorkItem* items, int n_items, int* counter,
                              int g, int blocks, bool ragged, cudaStream_t st);

// float-float dipole path (bpm_dipole_ff.cu): position digits and moment
// pairs of every particle, then the symmetric all-pairs kernel
cudaError_t launch_ff_encode(const Sys& s, cudaStream_t st);
// Sets a kernel's dynamic shared memory limit to the device's (once for all
// handles); true when smem bytes fit.
bool allow_dynamic_smem(const void* fn, size_t smem);
int dipole_ff_tile();
int dipole_ff_blocks_per_sm(int g);
cudaError_t launch_dipole_sym_ff(const Sys& s, const WorkItem* items, int n_items, int* counter, int g, int blocks,
                                 bool ragged, cudaStream_t st);
// the symmetric dipole VJP of the adjoint in float-float (BPM_FF handles):
// encodes the snapshot's positions, m, lam, mu into a.ffbuf, then the pairs
int adj_ff_comp();
cudaError_t launch_adj_dipole_sym_ff(const Sys& s, const AdjBuf& a, int64_t n_items, cudaStream_t st);

// contact between non-bonded particles: rebuilds the cell list and adds the
// contact forces and torques to f, t (after the bond kernel)
cudaError_t launch_contact(const Sys& s, const Contact& c, cudaStream_t st);
int contact_scan_blocks(uint32_t H);  // scan scratch entries for H buckets

// fluid: init f = f_eq(rho0, u0); one LBM step from buffer `parity`;
// macroscopic fields; interpolation at the particles; penalty force and
// (time-stepping evaluations) its spread reaction
cudaError_t launch_lbm_init(const Lbm& L, const double* rho0, const double* u0, cudaStream_t st);
cudaError_t launch_lbm_step(const Lbm& L, int parity, cudaStream_t st);
cudaError_t launch_lbm_macro(const Lbm& L, int parity, double* rho, double* u, cudaStream_t st);
cudaError_t launch_ibm_interp(const Sys& s, const Lbm& L, int parity, cudaStream_t st);
cudaError_t launch_ibm_penalty(const Sys& s, const Lbm& L, cudaStream_t st);

// reduce dipole partials into f/t and advance the state
enum FinishMode : int { FINISH_FORCES = 0, FINISH_HALF_KICK = 1, FINISH_CONTINUE = 2 };
cudaError_t launch_finish(const Sys& s, bool dipole, int mode, bool energy, int* counter,
                          cudaStream_t st);
// sums each particle's partial slots into slot 0 (one thread per component
// and particle); the finish kernel then reads slot 0 only
cudaError_t launch_reduce_slots(const Sys& s, cudaStream_t st);
// first half kick + drift + Richardson update of the first step of a run
cudaError_t launch_first_half(const Sys& s, cudaStream_t st);
// deterministic reduction of the energy scratch into out[5] (device)
cudaError_t launch_energy_reduce(const Sys& s, double* out5, cudaStream_t st);

// AoS <-> SoA conversion; ncomp = 3 or 4
cudaError_t launch_aos_to_soa(const double* aos, double* soa, int64_t n, int ncomp, cudaStream_t st);
cudaError_t launch_soa_to_aos(const double* soa, double* aos, int64_t n, int ncomp, cudaStream_t st);
// state transforms used by set/get state (rest-orientation gauge)
cudaError_t launch_quat_right_mul(double* q_soa, const double* r_soa, int64_t n, bool conj_r,
                                  bool normalise, cudaStream_t st);
cudaError_t launch_zero_clamped(const Sys& s, cudaStream_t st);
// v <- q v q* (or q* v q when inverse) for SoA vectors and quaternions
cudaError_t launch_rotate_vec(const double* q_soa, double* v_soa, int64_t n, bool inverse,
                              cudaStream_t st);

// adjoint sweep (bpm_adjoint.cu)
cudaError_t launch_adj_phi(const Sys& s, const AdjBuf& a, int dipole_mode, const int64_t* rod_off,
                           cudaStream_t st);
cudaError_t launch_adj_update(const Sys& prev, const Sys& cur, const AdjBuf& a, double kick, cudaStream_t st);
cudaError_t launch_adj_reduce_B(const double* aB, int64_t n, double* out, cudaStream_t st);

}  // namespace bpm
