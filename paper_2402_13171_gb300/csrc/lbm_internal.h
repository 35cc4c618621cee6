// Internal descriptors shared by the CUDA kernels (lbm_kernels.cu) and the
// host runtime behind the C ABI (lbm_abi.cu).  Plain old data only: these
// structs are copied to device memory as they are.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_gb300.h"

namespace lbmgb {

constexpr int kMaxTurbines = 16;    // rotors per lattice
constexpr int kMaxElements = 4096;  // blade elements per lattice
constexpr int kMaxInstances = 64;   // lattices per batch
constexpr long long kDefaultWaitCycles = 1ll << 31;  // ~1 s of SM clock before a device wait is declared failed

enum Bc : int { BC_PERIODIC = 0, BC_INOUT = 1, BC_NOSLIP = 2, BC_FREESLIP = 3 };
enum Coll : int { COLL_CUMULANT = 0, COLL_SRT_SMAG = 1 };
enum Store : int { STORE_FP32 = 0, STORE_BF16 = 1, STORE_FP16 = 2 };

// Device error bits (DevDomain::err).
enum ErrBits : unsigned { ERR_NONFINITE = 1u, ERR_ELEMENT_OUTSIDE = 2u, ERR_TIMEOUT = 4u };

// One rotor.  Rotor basis: e_axis = (cos yaw, sin yaw, 0), e1 = (-sin yaw,
// cos yaw, 0), e2 = (0, 0, 1); blade direction e_r = cos(theta) e1 + sin(theta) e2.
struct DevTurbine {
    float hub[3];
    float radius;
    int n_blades, n_elements;
    float eps, inv_eps2, cut;  // Gaussian width, 1/eps^2, per-axis cut-off (3 eps, or 3/2 for Roma)
    int roma;                  // 1: Roma three-point delta, 0: Gaussian
    int tip_loss;              // 1: Glauert tip-loss factor on the element forces
    double omega, theta0;      // rad per step, rad
    float e_axis[3], e1[3], e2[3];
    float pitch, chord_root, chord_tip;
    const float* twist;        // n_elements or nullptr
    int n_polar;
    const float* alpha;
    const float* cl;
    const float* cd;
    int polar_uniform;         // alpha equally spaced: direct segment index
    float polar_a0, polar_inv_da;
    int lo[3], hi[3];          // force box, inclusive cell bounds
    int bnx, bny;              // box extents along x, y
    long long bcells;          // cells in the box
    float* fbox;               // ALM force of the last collision at the box cells, 3 planes
    int el_offset;             // first element of this rotor in the lattice's element list
};

// One lattice.
struct DevDomain {
    int nx, ny, nz;
    long long N;
    int bc[3];
    float omega;               // shear relaxation rate 1/(3 nu + 1/2)
    float tau0;                // 3 nu + 1/2
    float smag_c2;             // Smagorinsky C^2
    float body[3];
    int inflow_kind;           // 0 uniform, 1 log law
    double u_ref[3];
    double z0, inv_log_zref_z0;
    double noise_amp;          // noise_rel * |u_ref|
    unsigned long long seed;
    float u_ref_f[3], noise_amp_f;
    float* inflow_scale;       // nz: mean-profile factor per z plane (1, or the log law)
    float* inflow_ghost[2];    // by step parity: inlet ghost populations per column (x inlet only):
                               // [9][nz][ny] offsets feq_q(1, u_in) - w_q of the nine directions with
                               // c_x = +1, index (cz + 1) * 3 + (cy + 1)
    float* outlet[2];          // by step parity (in-place lattices with an x outlet only): the last plane's
                               // post-collision populations of the nine directions with c_x = -1,
                               // [9][nz][ny], index (cz + 1) * 3 + (cy + 1)
    void* f[2];                // PDF offset arrays [27][nz][ny][nx] of the storage type
    int n_turb;
    DevTurbine* turb;          // device array of n_turb
    float4* el_pos[2];         // by step parity: element position (xyz) and 1/(Sx Sy Sz) (w)
    float4* el_force[2];       // by step parity: blade force (xyz)
    double* el_load;           // scratch, 2 doubles per element
    double* loads[2];          // by step parity: thrust, torque per rotor
    double* loads_sink;        // mapped page-locked host ring, or nullptr: step s's loads at [(s % sink_len) n_turb + t] * 2
    int sink_len;
    int n_el;
    unsigned int* rotor_counter;  // CTAs of the actuator-line launch done (the last adds up the loads)
    int diag_every;
    double* diag_acc;          // 4 doubles, accumulated on a diagnostic step
    double* diag_res;          // 4 doubles + the step they belong to
    unsigned int* err;
};

// Arguments of one stream-collide launch over all lattices of a batch.
struct StepArgs {
    const DevDomain* dom;               // device array
    const unsigned long long* tiles;    // this launch's part of the work list (the rotor tiles, or the rest)
    unsigned int n_tiles;               // entries in that part
    unsigned int n_total;               // entries of the whole step (both launches): diagnostic close-out
    int write_step;                     // 1 for the launch of a step whose CTA 0 advances the step slot
    int n_inst;
    int parity;                         // source array f[parity], destination f[parity ^ 1]
    long long* step_slot;               // step n in slot [parity]; CTA 0 writes n+1 to slot [parity ^ 1]
    int* diag_flag;                     // slot [parity]: 1 if step n is a diagnostic step; CTA 0 writes n+1's
    unsigned int* diag_done;            // CTA completion counter, used on diagnostic steps only
    int diag_every;                     // diagnostic period shared by the batch (0 = off)
    int tile_z;                         // planes per CTA (1: no marching); for the rotor launch the deepest rotor tile
    int staged;                         // rows staged in shared memory by persistent CTAs
    long long wait_cycles;              // bound of the staged step's copy-barrier waits (SM clock cycles)
    int trigger;                        // a non-rotor launch followed by a dependent launch: let it start early
};

// Per-lattice values the bulk launch reads for every cell, passed in its
// kernel parameters (constant bank) rather than read from the descriptor.
struct LatHot {
    int nx, ny, nz;
    unsigned N;
    int inout;                 // x inlet/outlet (else periodic x)
    float omega, tau0, smag_c2;
    float body[3];
    void* f[2];
};
struct BulkParams {
    LatHot lat[kMaxInstances];
};

// Arguments of the actuator-line launch (k_alm): one CTA per block of
// kAlmBlock blade elements of each lattice, the last CTA of a lattice adding up
// its per-rotor FP64 loads.
constexpr int kAlmBlock = 32;
struct AlmArgs {
    const DevDomain* dom;               // device array
    int n_inst;
    int cta_off[kMaxInstances + 1];     // first CTA of each lattice; cta_off[n_inst] = grid size
    const long long* step_slot;         // in a time step: step n in slot [slot], the launch evaluates n + 1;
    int slot;                           //   nullptr: evaluate `step`
    long long step;
    int array;                          // PDF array read, f[array]
    int swapped;                        // in-place array after an even step: pulled values in the own opposite slots
};
// CTA offsets of the lattices for element counts n_el[0..n_inst); returns the grid size.
inline int alm_blocks(AlmArgs& a, const int* n_el, int n_inst)
{
    int c = 0;
    a.n_inst = n_inst;
    for (int i = 0; i < n_inst; ++i) {
        a.cta_off[i] = c;
        c += (n_el[i] + kAlmBlock - 1) / kAlmBlock;
    }
    a.cta_off[n_inst] = c;
    return c;
}

// Planes a rotor tile covers at most (consecutive z-blocks of its column are
// merged up to this depth), so that one CTA culls the blade elements once for
// several planes.
constexpr int kRotorPlanes = 3;

// Work-list entry: bit 63 rotor tile, bits 56..62 planes - 1 (rotor tiles),
// 48..55 lattice, 32..47 z, 16..31 y0, 0..15 x0.
__host__ __device__ inline unsigned long long pack_tile(int inst, int z, int y0, int x0, bool rotor, int planes = 1)
{
    return ((unsigned long long)(rotor ? 1u : 0u) << 63) | ((unsigned long long)((planes - 1) & 0x7F) << 56) |
           ((unsigned long long)(inst & 0xFF) << 48) | ((unsigned long long)(z & 0xFFFF) << 32) |
           ((unsigned long long)(y0 & 0xFFFF) << 16) | (unsigned long long)(x0 & 0xFFFF);
}
__host__ __device__ inline int tile_lattice(unsigned long long t) { return (int)((t >> 48) & 0xFF); }
__host__ __device__ inline int tile_planes(unsigned long long t) { return (int)((t >> 56) & 0x7F) + 1; }

// Host-side checks of a rotor description shared by alm_add_turbine and
// alm_eval_static: blade and element counts in [1, max_elements] each and their
// product at most max_elements (formed in 64 bits, so it cannot wrap), and every
// real-valued input finite (a NaN hub would pass the support test, whose
// comparisons are all false for NaN).
inline bool turbine_counts_ok(const alm_turbine_desc* d, long long max_elements)
{
    if (d->n_blades < 1 || d->n_elements < 1 || d->n_blades > max_elements || d->n_elements > max_elements) return false;
    return (long long)d->n_blades * (long long)d->n_elements <= max_elements;
}
inline bool turbine_values_finite(const alm_turbine_desc* d)
{
    const double v[] = {d->hub[0], d->hub[1], d->hub[2], d->radius, d->epsilon, d->omega, d->yaw, d->pitch,
                        d->theta0, d->chord_root, d->chord_tip};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    if (d->twist)
        for (int k = 0; k < d->n_elements; ++k)
            if (!std::isfinite(d->twist[k])) return false;
    for (int i = 0; i < d->n_polar; ++i)
        if (!std::isfinite(d->alpha[i]) || !std::isfinite(d->cl[i]) || !std::isfinite(d->cd[i])) return false;
    return true;
}

// Host-side launchers (lbm_kernels.cu).
// rotor: the launch over the rotor tiles (element culling, force gather, the
// actuator line of the next step) rather than over the rest.  dependent: a
// bulk launch that directly follows its own step's rotor launch on the stream
// and may overlap it (programmatic stream serialization).
// bulk: the lattices' per-cell parameters for the bulk kernel over the tiles
// without a wall-face cell (nullptr: the general kernel); diag_step: the step is a
// diagnostic step (the bulk kernel then carries the FP64 sums; the general
// kernels read the step's diagnostic flag on the device); pairs: the bulk kernel
// takes two cells of a row per thread (16-bit storage, every nx even), its block
// (block.x / 2, block.y) over the same tiles.
cudaError_t launch_step(int coll, int store, dim3 grid, dim3 block, cudaStream_t s, const StepArgs& a, bool rotor,
                        bool dependent, const BulkParams* bulk = nullptr, bool diag_step = false, bool pairs = false);
// The in-place (AA) step over the whole work list: odd steps read and write a
// cell's own slots, even steps pull and push across neighbours.
// rotor / dependent as for launch_step; pairs (the lattices' per-cell
// parameters, or nullptr): tiles without a wall-face cell, two cells of a row
// per thread (16-bit storage, every nx even).
cudaError_t launch_step_aa(int coll, int store, dim3 grid, dim3 block, cudaStream_t s, const StepArgs& a, bool odd,
                           bool rotor, bool dependent, const BulkParams* pairs = nullptr);
// Outlet copies of an in-place lattice for step `step`, from its current state.
cudaError_t launch_outlet_fill(int store, const DevDomain* d_dom_inst, const DevDomain& h, long long step,
                               cudaStream_t s);
// The actuator line (k_alm over alm_blocks' grid).  dependent: launched right
// after its step's rotor launch, which it waits for on the device while the
// launches after it may already start (programmatic stream serialization).
cudaError_t launch_alm(int store, const AlmArgs& a, cudaStream_t s, bool dependent);
int staged_blocks_per_sm(int coll, int store, int width);
cudaError_t launch_inflow(const DevDomain* d_dom_inst, const DevDomain& h, long long step, cudaStream_t s);
cudaError_t launch_init(int store, const DevDomain* d_dom_inst, const DevDomain& h, const double* rho,
                        const double* u, const float* fneq, int parity, int inflow_mean, cudaStream_t s);
cudaError_t launch_moments(int store, const DevDomain* d_dom_inst, const DevDomain& h, int parity, double* rho,
                           double* u, cudaStream_t s);
cudaError_t launch_probe(int store, const DevDomain* d_dom_inst, int parity, const long long* cells, int n, double* out,
                         cudaStream_t s);
// One PDF plane of n values as FP64 populations w + h, and back.
cudaError_t launch_plane_to_f64(int store, const void* src, double* dst, long long n, double w, cudaStream_t s);
cudaError_t launch_plane_from_f64(int store, const double* src, void* dst, long long n, double w, cudaStream_t s);

}  // namespace lbmgb
