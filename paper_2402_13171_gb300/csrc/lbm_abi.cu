// Host runtime behind the C ABI of include/lbm_gb300.h: lattice contexts and
// batches, device memory, the per-step work list (rotor tiles first), CUDA
// graph replay of the single-launch time step, state input/output, and error
// reporting.  All compute runs in the kernels of lbm_kernels.cu.
#include "lbm_gb300.h"
#include "lbm_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace lbmgb;

namespace {

struct TurbineHost {
    alm_turbine_desc desc{};
    std::vector<double> twist, alpha, cl, cd;
    DevTurbine dev{};
};

struct Instance {
    lbm_config cfg{};
    DevDomain h{};
    std::vector<TurbineHost> turb;
    DevTurbine* d_turb = nullptr;
    unsigned char* small = nullptr;  // counters, diagnostics, error flags
};

struct Batch {
    int refs = 0;
    std::vector<Instance> inst;
    int coll = 0, store = 0;
    cudaStream_t stream = nullptr;
    void* (*ualloc)(size_t, void*) = nullptr;
    void (*ufree)(void*, void*) = nullptr;
    void* user = nullptr;
    std::vector<void*> allocs;
    DevDomain* d_dom = nullptr;
    unsigned long long* d_tiles = nullptr;
    size_t tiles_cap = 0;
    unsigned n_tiles = 0;
    long long* d_step = nullptr;          // two slots: step n lives in slot [n & 1]
    int* d_diag_flag = nullptr;           // two slots: 1 if step n is a diagnostic step
    unsigned int* d_diag_done = nullptr;
    int host_diag_flag = 0;
    int diag_every = 0;
    long long host_step = 0;
    int tile_x = 32, tile_y = 4, tile_z = 1;
    int staged = 0;        // rows staged in shared memory by persistent CTAs
    unsigned staged_grid = 0;
    int single_cell = 0;   // the bulk launch keeps one cell per thread where pairs would apply
    bool pairs_ok = false; // 16-bit storage and every nx even: paired bulk cells
    lbm_status status = LBM_OK;
    std::string err;
    bool dirty = true;
    bool profiling = false;
    std::vector<cudaEvent_t> ev;         // pairs bracketing timed launches
    std::vector<int> ev_launches;        // step launches inside each pair
    size_t ev_used = 0;
    double prof_ms = 0.0;
    long long prof_n = 0;
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [long?][start parity]
    unsigned n_rotor = 0;                 // rotor tiles at the head of the work list
    unsigned n_face = 0;                  // then the tiles with a no-slip or free-slip face cell
    int rotor_planes = 1;                 // planes of the deepest rotor tile
    int inplace = 0;                      // one PDF array, AA pattern
    long long* d_probe = nullptr;   // probe cell list and results, grown on demand
    double* d_probe_out = nullptr;
    int probe_cap = 0;
    void* d_stage = nullptr;        // staging for host input/output, grown on demand and reused
    size_t stage_cap = 0;
    long long wait_cycles = kDefaultWaitCycles;  // bound of the staged step's copy-barrier waits
};

}  // namespace

struct lbm_ctx {
    Batch* b;
    int idx;
};

namespace {

size_t store_bytes(int s) { return s == STORE_FP32 ? 4 : 2; }

double w1h(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
double wqh(int q) { return w1h(q % 3 - 1) * w1h((q / 3) % 3 - 1) * w1h(q / 9 - 1); }

lbm_status fail(Batch* b, lbm_status s, const std::string& msg, bool sticky = true)
{
    b->err = msg;
    if (sticky && b->status == LBM_OK) b->status = s;
    return s;
}

#define CK(x)                                                                                         \
    do {                                                                                              \
        cudaError_t e_ = (x);                                                                         \
        if (e_ != cudaSuccess) return fail(b, LBM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// NVTX range over a host call, for timeline profilers (free when none is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Host-side fault injection for tests of the error paths; nothing reaches the
// GPU.  LBM_FAULT=alloc fails every device allocation, =capture every graph
// capture, =step:N the lbm_step call that would run step N.  Read at each
// check, so a process can set and clear it between calls.
const char* injected_fault(const char* what)
{
    const char* f = std::getenv("LBM_FAULT");
    if (!f) return nullptr;
    const size_t n = std::strlen(what);
    if (std::strncmp(f, what, n) != 0 || (f[n] != '\0' && f[n] != ':')) return nullptr;
    return f + n;
}

void* dalloc(Batch* b, size_t bytes)
{
    void* p = nullptr;
    if (injected_fault("alloc")) return nullptr;
    if (bytes == 0) bytes = 16;
    if (b->ualloc) {
        p = b->ualloc(bytes, b->user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) b->allocs.push_back(p);
    return p;
}

void dfree(Batch* b, void* p)
{
    if (!p) return;
    auto it = std::find(b->allocs.begin(), b->allocs.end(), p);
    if (it != b->allocs.end()) b->allocs.erase(it);
    if (b->ufree) b->ufree(p, b->user);
    else cudaFree(p);
}

void drop_graphs(Batch* b)
{
    for (auto& row : b->gexec)
        for (auto& g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

void destroy_batch(Batch* b)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    drop_graphs(b);
    for (auto e : b->ev) cudaEventDestroy(e);
    std::vector<void*> all = b->allocs;
    for (void* p : all) dfree(b, p);
    delete b;
}

lbm_status validate_cfg(const lbm_config* c, std::string& msg)
{
    if (!c) { msg = "null config"; return LBM_ERR_INVALID_ARG; }
    if (c->nx < 1 || c->ny < 1 || c->nz < 1 || c->nx > 65535 || c->ny > 65535 || c->nz > 65535) {
        msg = "lattice sizes must be in [1, 65535]";
        return LBM_ERR_INVALID_ARG;
    }
    if ((long long)c->nx * c->ny * c->nz * 27LL >= (1LL << 31)) {
        msg = "lattice too large: 27 * nx * ny * nz must stay below 2^31 (79,536,431 cells)";
        return LBM_ERR_INVALID_ARG;
    }
    if (c->collision != LBM_COLL_CUMULANT && c->collision != LBM_COLL_SRT_SMAGORINSKY) {
        msg = "unknown collision";
        return LBM_ERR_INVALID_ARG;
    }
    if (c->storage < 0 || c->storage > 2) { msg = "unknown storage"; return LBM_ERR_INVALID_ARG; }
    if (!(c->nu > 0.0) || !std::isfinite(c->nu)) { msg = "nu must be > 0"; return LBM_ERR_INVALID_ARG; }
    for (int a = 0; a < 3; ++a) {
        if (c->bc[a] < 0 || c->bc[a] > 3) { msg = "unknown boundary code"; return LBM_ERR_INVALID_ARG; }
        if (a > 0 && c->bc[a] == LBM_BC_INFLOW_OUTFLOW) { msg = "inflow/outflow is x only"; return LBM_ERR_INVALID_ARG; }
    }
    if (c->bc[0] == LBM_BC_INFLOW_OUTFLOW && c->nx < 2) { msg = "inflow/outflow needs nx >= 2"; return LBM_ERR_INVALID_ARG; }
    if (c->diag_every < 0) { msg = "diag_every must be >= 0"; return LBM_ERR_INVALID_ARG; }
    const int tx = c->tile_x ? c->tile_x : 32, ty = c->tile_y ? c->tile_y : 4, tz = c->tile_z ? c->tile_z : 1;
    if (tx < 32 || tx % 32 != 0 || ty < 1 || tx * ty > 256 || tz < 1 || tz > 64) {
        msg = "tile_x must be a multiple of 32, tile_x * tile_y <= 256, 1 <= tile_z <= 64";
        return LBM_ERR_INVALID_ARG;
    }
    if (c->inplace != 0 && c->inplace != 1) { msg = "inplace must be 0 or 1"; return LBM_ERR_INVALID_ARG; }
    if (c->staged < 0 || c->staged > 2) { msg = "staged must be 0, 1 or 2"; return LBM_ERR_INVALID_ARG; }
    if (c->inplace) {
        if (tz != 1 || c->staged == 1) {
            msg = "the in-place scheme takes single-plane direct tiles only";
            return LBM_ERR_UNSUPPORTED;
        }
    }
    return LBM_OK;
}

lbm_status init_instance(Batch* b, Instance& I, const lbm_config& c)
{
    I.cfg = c;
    DevDomain& h = I.h;
    h.nx = c.nx;
    h.ny = c.ny;
    h.nz = c.nz;
    h.N = (long long)c.nx * c.ny * c.nz;
    for (int a = 0; a < 3; ++a) {
        h.bc[a] = c.bc[a];
        h.body[a] = (float)c.body_force[a];
        h.u_ref[a] = 0.0;
    }
    h.tau0 = (float)(3.0 * c.nu + 0.5);
    h.omega = (float)(1.0 / (3.0 * c.nu + 0.5));
    h.smag_c2 = (float)(c.smag_c * c.smag_c);
    h.inflow_kind = 0;
    h.z0 = 0.1;
    h.inv_log_zref_z0 = 1.0;
    h.noise_amp = 0.0;
    h.noise_amp_f = 0.0f;
    h.u_ref_f[0] = h.u_ref_f[1] = h.u_ref_f[2] = 0.0f;
    h.seed = c.seed;
    h.inflow_scale = (float*)dalloc(b, sizeof(float) * c.nz);
    if (!h.inflow_scale) return fail(b, LBM_ERR_OOM, "inflow table allocation failed");
    {
        std::vector<float> ones(c.nz, 1.0f);
        CK(cudaMemcpyAsync(h.inflow_scale, ones.data(), sizeof(float) * c.nz, cudaMemcpyHostToDevice, b->stream));
        if (b->stream) CK(cudaStreamSynchronize(b->stream));
    }
    h.inflow_ghost[0] = h.inflow_ghost[1] = nullptr;
    if (c.bc[0] == LBM_BC_INFLOW_OUTFLOW) {
        const size_t ib = sizeof(float) * 9 * (size_t)c.ny * c.nz;
        float* g2 = (float*)dalloc(b, 2 * ib);
        if (!g2) return fail(b, LBM_ERR_OOM, "inflow buffer allocation failed");
        CK(cudaMemsetAsync(g2, 0, 2 * ib, b->stream));
        h.inflow_ghost[0] = g2;
        h.inflow_ghost[1] = g2 + 9 * (size_t)c.ny * c.nz;
    }
    h.outlet[0] = h.outlet[1] = nullptr;
    if (c.inplace && c.bc[0] == LBM_BC_INFLOW_OUTFLOW) {
        const size_t ob = sizeof(float) * 9 * (size_t)c.ny * c.nz;
        float* o2 = (float*)dalloc(b, 2 * ob);
        if (!o2) return fail(b, LBM_ERR_OOM, "outlet buffer allocation failed");
        CK(cudaMemsetAsync(o2, 0, 2 * ob, b->stream));
        h.outlet[0] = o2;
        h.outlet[1] = o2 + 9 * (size_t)c.ny * c.nz;
    }
    const size_t fbytes = (size_t)h.N * 27 * store_bytes(b->store);
    for (int p = 0; p < (c.inplace ? 1 : 2); ++p) {
        h.f[p] = dalloc(b, fbytes);
        if (!h.f[p]) return fail(b, LBM_ERR_OOM, "PDF array allocation failed");
        CK(cudaMemsetAsync(h.f[p], 0, fbytes, b->stream));  // offsets 0: f = w, the rest state
    }
    if (c.inplace) h.f[1] = h.f[0];  // one array: both parities name it
    I.d_turb = (DevTurbine*)dalloc(b, sizeof(DevTurbine) * kMaxTurbines);
    void* ep = dalloc(b, sizeof(float4) * kMaxElements * 4);
    void* el = dalloc(b, sizeof(double) * 2 * kMaxElements);
    void* ld = dalloc(b, sizeof(double) * 4 * kMaxTurbines);
    I.small = (unsigned char*)dalloc(b, 256);
    if (!I.d_turb || !ep || !el || !ld || !I.small) return fail(b, LBM_ERR_OOM, "descriptor allocation failed");
    CK(cudaMemsetAsync(ep, 0, sizeof(float4) * kMaxElements * 4, b->stream));
    CK(cudaMemsetAsync(el, 0, sizeof(double) * 2 * kMaxElements, b->stream));
    CK(cudaMemsetAsync(ld, 0, sizeof(double) * 4 * kMaxTurbines, b->stream));
    CK(cudaMemsetAsync(I.small, 0, 256, b->stream));
    float4* e4 = (float4*)ep;
    h.el_pos[0] = e4;
    h.el_pos[1] = e4 + kMaxElements;
    h.el_force[0] = e4 + 2 * kMaxElements;
    h.el_force[1] = e4 + 3 * kMaxElements;
    h.el_load = (double*)el;
    h.loads[0] = (double*)ld;
    h.loads[1] = (double*)ld + 2 * kMaxTurbines;
    h.diag_acc = (double*)I.small;             // 4 doubles
    h.diag_res = (double*)I.small + 4;         // 5 doubles
    h.rotor_counter = (unsigned int*)(I.small + 128);
    h.err = (unsigned int*)(I.small + 132);
    h.turb = I.d_turb;
    h.n_turb = 0;
    h.n_el = 0;
    h.diag_every = c.diag_every;
    return LBM_OK;
}

// Upload descriptors and rebuild the work list: rotor tiles of every lattice first.
lbm_status sync_descriptors(Batch* b)
{
    if (!b->dirty) return LBM_OK;
    std::vector<unsigned long long> rotor, face, rest;
    // rotor tiles: the z-blocks of a column that reach a rotor box, runs of them
    // merged up to kRotorPlanes planes (not for the staged kernel's row segments)
    const int merge = b->staged ? 1 : std::max(1, kRotorPlanes / b->tile_z);
    int rotor_planes = 1;
    for (size_t i = 0; i < b->inst.size(); ++i) {
        Instance& I = b->inst[i];
        const int nzb = (I.h.nz + b->tile_z - 1) / b->tile_z;
        const int nyb = (I.h.ny + b->tile_y - 1) / b->tile_y, nxb = (I.h.nx + b->tile_x - 1) / b->tile_x;
        // planes[(k * nyb + j) * nxb + l]: 0 for a bulk tile, -1 for a z-block inside a
        // merged rotor tile that starts below it, else the rotor tile's planes
        std::vector<int> planes((size_t)nzb * nyb * nxb, 0);
        for (int j = 0; j < nyb; ++j)
            for (int l = 0; l < nxb; ++l) {
                const int y0 = j * b->tile_y, x0 = l * b->tile_x;
                auto hit = [&](int k) {
                    const int z = k * b->tile_z;
                    for (auto& t : I.turb) {
                        const DevTurbine& B = t.dev;
                        if (z <= B.hi[2] && z + b->tile_z - 1 >= B.lo[2] && y0 <= B.hi[1] &&
                            y0 + b->tile_y - 1 >= B.lo[1] && x0 <= B.hi[0] && x0 + b->tile_x - 1 >= B.lo[0])
                            return true;
                    }
                    return false;
                };
                for (int k = 0; k < nzb;) {
                    if (!hit(k)) {
                        ++k;
                        continue;
                    }
                    int run = 1;
                    while (run < merge && k + run < nzb && hit(k + run)) ++run;
                    planes[((size_t)k * nyb + j) * nxb + l] = std::min(run * b->tile_z, I.h.nz - k * b->tile_z);
                    for (int r = 1; r < run; ++r) planes[((size_t)(k + r) * nyb + j) * nxb + l] = -1;
                    k += run;
                }
            }
        // z-major order (x fastest), as the bulk streams plane after plane
        for (int k = 0; k < nzb; ++k)
            for (int j = 0; j < nyb; ++j)
                for (int l = 0; l < nxb; ++l) {
                    const int p = planes[((size_t)k * nyb + j) * nxb + l];
                    const int z = k * b->tile_z, y0 = j * b->tile_y, x0 = l * b->tile_x;
                    if (p == 0) {
                        // a cell of the tile on a no-slip or free-slip face: the general kernel
                        const int lo[3] = {x0, y0, z}, ext[3] = {b->tile_x, b->tile_y, b->tile_z};
                        const int n3[3] = {I.h.nx, I.h.ny, I.h.nz};
                        bool on_face = false;
                        for (int a3 = 0; a3 < 3; ++a3)
                            if ((I.h.bc[a3] == BC_NOSLIP || I.h.bc[a3] == BC_FREESLIP) &&
                                (lo[a3] == 0 || lo[a3] + ext[a3] - 1 >= n3[a3] - 1))
                                on_face = true;
                        (on_face ? face : rest).push_back(pack_tile((int)i, z, y0, x0, false));
                    } else if (p > 0) {
                        rotor.push_back(pack_tile((int)i, z, y0, x0, true, p));
                        rotor_planes = std::max(rotor_planes, p);
                    }
                }
        std::vector<DevTurbine> dt;
        for (auto& t : I.turb) dt.push_back(t.dev);
        if (!dt.empty())
            CK(cudaMemcpyAsync(I.d_turb, dt.data(), sizeof(DevTurbine) * dt.size(), cudaMemcpyHostToDevice, b->stream));
    }
    std::vector<unsigned long long> tiles = rotor;
    tiles.insert(tiles.end(), face.begin(), face.end());
    tiles.insert(tiles.end(), rest.begin(), rest.end());
    if (tiles.size() > b->tiles_cap) {
        if (b->d_tiles) dfree(b, b->d_tiles);
        b->tiles_cap = 0;
        b->d_tiles = (unsigned long long*)dalloc(b, sizeof(unsigned long long) * tiles.size());
        if (!b->d_tiles) return fail(b, LBM_ERR_OOM, "work list allocation failed");
        b->tiles_cap = tiles.size();
    }
    b->n_tiles = (unsigned)tiles.size();
    b->n_rotor = (unsigned)rotor.size();
    b->n_face = (unsigned)face.size();
    b->rotor_planes = rotor_planes;
    CK(cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(unsigned long long) * tiles.size(), cudaMemcpyHostToDevice,
                       b->stream));
    std::vector<DevDomain> doms;
    for (auto& I : b->inst) doms.push_back(I.h);
    CK(cudaMemcpyAsync(b->d_dom, doms.data(), sizeof(DevDomain) * doms.size(), cudaMemcpyHostToDevice, b->stream));
    // pageable copies above are staged before returning; the stream orders them before any launch
    drop_graphs(b);
    b->dirty = false;
    return LBM_OK;
}

StepArgs step_args(Batch* b, int parity)
{
    StepArgs a;
    a.dom = b->d_dom;
    a.tiles = b->d_tiles;
    a.n_tiles = b->n_tiles;
    a.n_total = b->n_tiles;
    a.write_step = 1;
    a.n_inst = (int)b->inst.size();
    a.parity = parity;
    a.step_slot = b->d_step;
    a.diag_flag = b->d_diag_flag;
    a.diag_done = b->d_diag_done;
    a.diag_every = b->diag_every;
    a.tile_z = b->tile_z;
    a.staged = b->staged;
    a.wait_cycles = b->wait_cycles;
    a.trigger = 0;
    return a;
}

// Step counter and diagnostic flag of host_step into their device slots.
cudaError_t write_step_slot(Batch* b)
{
    const int slot = (int)(b->host_step & 1);
    b->host_diag_flag = b->diag_every > 0 && b->host_step % b->diag_every == 0;
    cudaError_t e = cudaMemcpyAsync(b->d_step + slot, &b->host_step, sizeof(long long), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_diag_flag + slot, &b->host_diag_flag, sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && b->stream) e = cudaStreamSynchronize(b->stream);
    return e;
}

// Arguments of the actuator-line launch over every lattice with blade
// elements: of step n+1 inside the time step n (step read from the device slot
// `slot`, the array and layout the step leaves), or of the step `step` on the
// current array (refresh after a state change).
AlmArgs alm_args(Batch* b, const long long* step_slot, int slot, long long step, int array, int swapped)
{
    AlmArgs a{};
    a.dom = b->d_dom;
    int n_el[kMaxInstances];
    for (size_t i = 0; i < b->inst.size(); ++i) n_el[i] = b->inst[i].h.n_el;
    alm_blocks(a, n_el, (int)b->inst.size());
    a.step_slot = step_slot;
    a.slot = slot;
    a.step = step;
    a.array = array;
    a.swapped = swapped;
    return a;
}

// Two cells of a row per thread: 16-bit storage, every nx even, not the
// one-cell form, and CTAs of whole warps (tile_x * tile_y / 2 threads a
// multiple of 32, for the warp-wide reductions).
static bool pair_tiles(const Batch* b)
{
    return b->pairs_ok && !b->single_cell && (b->tile_x * b->tile_y) % 64 == 0;
}

// Per-lattice values the bulk kernels take as kernel parameters (constant bank)
// instead of loading them from the device descriptors.
static BulkParams bulk_params(const Batch* b)
{
    BulkParams bp{};
    for (size_t i = 0; i < b->inst.size(); ++i) {
        const DevDomain& h = b->inst[i].h;
        LatHot& L = bp.lat[i];
        L.nx = h.nx;
        L.ny = h.ny;
        L.nz = h.nz;
        L.N = (unsigned)h.N;
        L.inout = h.bc[0] == BC_INOUT ? 1 : 0;
        L.omega = h.omega;
        L.tau0 = h.tau0;
        L.smag_c2 = h.smag_c2;
        for (int a3 = 0; a3 < 3; ++a3) L.body[a3] = h.body[a3];
        L.f[0] = h.f[0];
        L.f[1] = h.f[1];
    }
    return bp;
}

// One time step.  Staged rows: one persistent launch over the whole work list,
// then (with rotors) the actuator line of the next step.  Otherwise (k_step or,
// in place, k_step_aa) the rotor tiles (first in the list), the actuator line
// of the next step (k_alm, which waits for them on the device), then the rest,
// allowed to overlap both; the step counter is advanced by the last launch.
// diag_step: the step is a diagnostic step (never inside a captured graph).
lbm_status launch_one(Batch* b, int parity, bool diag_step = false)
{
    const StepArgs a = step_args(b, parity);
    const dim3 block(b->tile_x, b->tile_y);
    if (b->staged) {
        CK(launch_step(b->coll, b->store, dim3(std::min(b->n_tiles, b->staged_grid)), block, b->stream, a, false,
                       false));
        if (b->n_rotor > 0)  // the actuator line of the next step, after it
            CK(launch_alm(b->store, alm_args(b, b->d_step, parity, 0, parity ^ 1, 0), b->stream, false));
        return LBM_OK;
    }
    const unsigned R = b->n_rotor, Nf = b->n_face, Np = b->n_tiles - b->n_rotor - b->n_face;
    if (b->inplace) {
        // the in-place kernels take every rule themselves: rotor tiles, then the rest
        const unsigned Nb = Nf + Np;
        StepArgs ar = a, ab = a;
        ar.n_tiles = R;
        ar.write_step = Nb == 0 ? 1 : 0;
        ab.tiles = b->d_tiles + R;
        ab.n_tiles = Nb;
        if (R > 0) {
            CK(launch_step_aa(b->coll, b->store, dim3(R), block, b->stream, ar, parity == 1, true, false));
            // after an even step the pulled populations of a cell are its own opposite slots
            CK(launch_alm(b->store, alm_args(b, b->d_step, parity, 0, 0, parity == 1 ? 0 : 1), b->stream, true));
        }
        if (!pair_tiles(b)) {
            if (Nb > 0) CK(launch_step_aa(b->coll, b->store, dim3(Nb), block, b->stream, ab, parity == 1, false, R > 0));
            return LBM_OK;
        }
        // 16-bit storage: the tiles with a wall-face cell one cell per thread, the
        // rest two cells per thread
        StepArgs af = ab, ap = ab;
        af.n_tiles = Nf;
        af.write_step = Np == 0 ? 1 : 0;
        ap.tiles = b->d_tiles + R + Nf;
        ap.n_tiles = Np;
        if (Nf > 0) CK(launch_step_aa(b->coll, b->store, dim3(Nf), block, b->stream, af, parity == 1, false, R > 0));
        if (Np > 0) {
            const BulkParams bp = bulk_params(b);
            CK(launch_step_aa(b->coll, b->store, dim3(Np), block, b->stream, ap, parity == 1, false, R + Nf > 0, &bp));
        }
        return LBM_OK;
    }
    // rotor tiles and the actuator line, then the face tiles (the general
    // kernel), then the plain bulk (k_bulk); each launch may start while the one
    // before still runs, the last one advances the step counter
    StepArgs ar = a, af = a, ap = a;
    ar.n_tiles = R;
    ar.write_step = (Nf + Np) == 0 ? 1 : 0;
    ar.tile_z = b->rotor_planes;  // > 1: the marching rotor kernel, each tile over its own planes
    af.tiles = b->d_tiles + R;
    af.n_tiles = Nf;
    af.write_step = Np == 0 ? 1 : 0;
    af.trigger = Np > 0 ? 1 : 0;
    ap.tiles = b->d_tiles + R + Nf;
    ap.n_tiles = Np;
    if (R > 0) {
        CK(launch_step(b->coll, b->store, dim3(R), block, b->stream, ar, true, false));
        CK(launch_alm(b->store, alm_args(b, b->d_step, parity, 0, parity ^ 1, 0), b->stream, true));
    }
    if (Nf > 0) CK(launch_step(b->coll, b->store, dim3(Nf), block, b->stream, af, false, R > 0));
    if (Np > 0) {
        const BulkParams bp = bulk_params(b);
        const bool tiled = b->tile_z == 1;  // k_bulk takes single-plane tiles
        const bool pairs = tiled && pair_tiles(b);
        CK(launch_step(b->coll, b->store, dim3(Np), block, b->stream, ap, false, R + Nf > 0, tiled ? &bp : nullptr,
                       diag_step, pairs));
    }
    return LBM_OK;
}

// Inlet velocities and actuator line of the current step for every lattice
// (after a state change).
lbm_status refresh_alm(Batch* b)
{
    lbm_status s = sync_descriptors(b);
    if (s != LBM_OK) return s;
    for (size_t i = 0; i < b->inst.size(); ++i) {
        if (b->inst[i].h.bc[0] == BC_INOUT) CK(launch_inflow(b->d_dom + i, b->inst[i].h, b->host_step, b->stream));
        if (b->inst[i].h.outlet[0])
            CK(launch_outlet_fill(b->store, b->d_dom + i, b->inst[i].h, b->host_step, b->stream));
    }
    bool any = false;
    for (auto& I : b->inst) any = any || I.h.n_el > 0;
    if (!any) return LBM_OK;
    CK(launch_alm(b->store, alm_args(b, nullptr, 0, b->host_step, (int)(b->host_step & 1), 0), b->stream, false));
    return LBM_OK;
}

lbm_status zero_fbox(Batch* b, Instance& I)
{
    for (auto& t : I.turb) CK(cudaMemsetAsync(t.dev.fbox, 0, sizeof(float) * 3 * t.dev.bcells, b->stream));
    return LBM_OK;
}

// Device staging buffer of at least `bytes` (> 0), reused across calls (stream-ordered).
void* stage(Batch* b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (bytes > b->stage_cap) {
        if (b->d_stage) dfree(b, b->d_stage);
        b->stage_cap = 0;
        b->d_stage = dalloc(b, bytes);
        if (!b->d_stage) return nullptr;
        b->stage_cap = bytes;
    }
    return b->d_stage;
}

lbm_status check_device_errors(Batch* b)
{
    if (b->stream) CK(cudaStreamSynchronize(b->stream));
    else CK(cudaDeviceSynchronize());
    for (auto& I : b->inst) {
        unsigned e = 0;
        CK(cudaMemcpy(&e, I.h.err, sizeof e, cudaMemcpyDeviceToHost));
        if (e & ERR_NONFINITE) return fail(b, LBM_ERR_NUMERIC, "non-finite mass or momentum in the diagnostic sums");
        if (e & ERR_ELEMENT_OUTSIDE) return fail(b, LBM_ERR_STATE, "a blade element left the lattice interior");
        if (e & ERR_TIMEOUT) return fail(b, LBM_ERR_TIMEOUT, "a bounded wait of the staged step gave up");
    }
    return LBM_OK;
}

lbm_status create_batch(int n, const lbm_config* cfgs, lbm_ctx** out)
{
    if (!out || n < 1 || n > kMaxInstances) return LBM_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        std::string msg;
        const lbm_status v = validate_cfg(cfgs + i, msg);
        if (v != LBM_OK) return v;
        if (cfgs[i].collision != cfgs[0].collision || cfgs[i].storage != cfgs[0].storage ||
            cfgs[i].inplace != cfgs[0].inplace ||
            cfgs[i].cuda_stream != cfgs[0].cuda_stream || cfgs[i].tile_x != cfgs[0].tile_x ||
            cfgs[i].tile_y != cfgs[0].tile_y || cfgs[i].tile_z != cfgs[0].tile_z ||
            cfgs[i].diag_every != cfgs[0].diag_every)
            return LBM_ERR_UNSUPPORTED;
    }
    Batch* b = new Batch();
    b->coll = cfgs[0].collision;
    b->store = cfgs[0].storage;
    b->stream = (cudaStream_t)cfgs[0].cuda_stream;
    b->ualloc = cfgs[0].dev_alloc;
    b->ufree = cfgs[0].dev_free;
    b->user = cfgs[0].alloc_user;
    b->tile_x = cfgs[0].tile_x ? cfgs[0].tile_x : 32;
    b->tile_y = cfgs[0].tile_y ? cfgs[0].tile_y : 4;
    b->tile_z = cfgs[0].tile_z ? cfgs[0].tile_z : 1;
    b->staged = 0;
    b->inplace = cfgs[0].inplace;
    const int want_staged = cfgs[0].staged;
    b->single_cell = want_staged == 2 ? 1 : 0;
    b->pairs_ok = b->store != STORE_FP32;
    for (int i = 0; i < n; ++i)
        if (cfgs[i].nx % 2 != 0) b->pairs_ok = false;
    b->diag_every = cfgs[0].diag_every;
    b->inst.resize(n);
    lbm_status s = LBM_OK;
    for (int i = 0; i < n && s == LBM_OK; ++i) s = init_instance(b, b->inst[i], cfgs[i]);
    if (s == LBM_OK) {
        b->d_dom = (DevDomain*)dalloc(b, sizeof(DevDomain) * n);
        void* sc = dalloc(b, 64);
        if (!b->d_dom || !sc) s = LBM_ERR_OOM;
        else {
            b->d_step = (long long*)sc;
            b->d_diag_done = (unsigned int*)((char*)sc + 16);
            b->d_diag_flag = (int*)((char*)sc + 32);
            if (cudaMemsetAsync(sc, 0, 64, b->stream) != cudaSuccess || write_step_slot(b) != cudaSuccess)
                s = LBM_ERR_CUDA;
        }
    }
    if (s == LBM_OK) s = sync_descriptors(b);
    if (s == LBM_OK && b->stream) s = cudaStreamSynchronize(b->stream) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
    if (s != LBM_OK) {
        destroy_batch(b);
        return s;
    }
    for (int i = 0; i < n; ++i) {
        out[i] = new lbm_ctx;
        out[i]->b = b;
        out[i]->idx = i;
        b->refs++;
    }
    if (want_staged == 1) {
        const lbm_status st = lbm_set_tile(out[0], b->tile_x, b->tile_y, b->tile_z, 1);
        if (st != LBM_OK) {
            for (int i = 0; i < n; ++i) lbm_destroy(out[i]);
            return st;
        }
    }
    return LBM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------- ABI

extern "C" {

const char* lbm_status_string(lbm_status s)
{
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_INVALID_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "out of device memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_NUMERIC: return "non-finite state";
    case LBM_ERR_TIMEOUT: return "device wait timed out";
    case LBM_ERR_STATE: return "invalid state";
    case LBM_ERR_UNSUPPORTED: return "unsupported combination";
    }
    return "unknown status";
}

lbm_status lbm_create(const lbm_config* cfg, lbm_ctx** out) { return create_batch(1, cfg, out); }

lbm_status lbm_batch_create(int n, const lbm_config* cfgs, lbm_ctx** out)
{
    if (!cfgs) return LBM_ERR_INVALID_ARG;
    return create_batch(n, cfgs, out);
}

void lbm_destroy(lbm_ctx* ctx)
{
    if (!ctx) return;
    Batch* b = ctx->b;
    delete ctx;
    if (--b->refs == 0) destroy_batch(b);
}

const char* lbm_last_error(const lbm_ctx* ctx)
{
    if (!ctx) return "null context";
    return ctx->b->err.c_str();
}

#define ENTER(ctx)                                    \
    if (!(ctx)) return LBM_ERR_INVALID_ARG;           \
    Batch* b = (ctx)->b;                              \
    Instance& I = b->inst[(ctx)->idx];                \
    (void)I;                                          \
    if (b->status != LBM_OK) return b->status;

// In-place lattices hold the two-array state only after an even number of steps.
#define REQUIRE_EVEN_STEP()                                                                                  \
    if (b->inplace && (b->host_step & 1))                                                                    \
        return fail(b, LBM_ERR_STATE, "in-place lattice: state access needs an even step count", false);

lbm_status lbm_set_inflow(lbm_ctx* ctx, const lbm_inflow* in)
{
    ENTER(ctx);
    REQUIRE_EVEN_STEP();
    if (!in || (in->kind != 0 && in->kind != 1)) return fail(b, LBM_ERR_INVALID_ARG, "bad inflow", false);
    if (in->kind == 1 && !(in->z0 > 0.0 && in->z_ref > in->z0))
        return fail(b, LBM_ERR_INVALID_ARG, "log law needs 0 < z0 < z_ref", false);
    for (int a = 0; a < 3; ++a) I.h.u_ref[a] = in->u_ref[a];
    I.h.inflow_kind = in->kind;
    I.h.z0 = in->kind == 1 ? in->z0 : 0.1;
    I.h.inv_log_zref_z0 = in->kind == 1 ? 1.0 / std::log(in->z_ref / in->z0) : 1.0;
    const double U0 = std::sqrt(in->u_ref[0] * in->u_ref[0] + in->u_ref[1] * in->u_ref[1] + in->u_ref[2] * in->u_ref[2]);
    I.h.noise_amp = in->noise_rel * U0;
    I.h.noise_amp_f = (float)I.h.noise_amp;
    for (int a = 0; a < 3; ++a) I.h.u_ref_f[a] = (float)in->u_ref[a];
    {
        std::vector<float> sc(I.h.nz, 1.0f);
        if (in->kind == 1)
            for (int z = 0; z < I.h.nz; ++z) sc[z] = (float)(std::log((z + 0.5) / in->z0) / std::log(in->z_ref / in->z0));
        CK(cudaMemcpyAsync(I.h.inflow_scale, sc.data(), sizeof(float) * I.h.nz, cudaMemcpyHostToDevice, b->stream));
        if (b->stream) CK(cudaStreamSynchronize(b->stream));
    }
    b->dirty = true;
    lbm_status s = sync_descriptors(b);
    if (s != LBM_OK) return s;
    const int par = (int)(b->host_step & 1);
    CK(launch_init(b->store, b->d_dom + ctx->idx, I.h, nullptr, nullptr, nullptr, par, 1, b->stream));
    s = zero_fbox(b, I);
    if (s != LBM_OK) return s;
    return refresh_alm(b);
}

lbm_status lbm_init_fields(lbm_ctx* ctx, const double* rho, const double* u, const float* fneq)
{
    NvtxRange nvtx_("lbm_init_fields");
    ENTER(ctx);
    REQUIRE_EVEN_STEP();
    const size_t N = (size_t)I.h.N;
    lbm_status s = sync_descriptors(b);
    if (s != LBM_OK) return s;
    // the caller's arrays go to the device as they are (FP64 rho, u; FP32 fneq)
    // and are converted there
    const size_t b_rho = rho ? 8 * N : 0, b_u = u ? 24 * N : 0, b_f = fneq ? 4 * 27 * N : 0;
    char* st = (char*)stage(b, b_rho + b_u + b_f);
    if (!st) return fail(b, LBM_ERR_OOM, "staging allocation failed");
    const double* d_rho = rho ? (const double*)st : nullptr;
    const double* d_u = u ? (const double*)(st + b_rho) : nullptr;
    const float* d_fneq = fneq ? (const float*)(st + b_rho + b_u) : nullptr;
    if (rho) CK(cudaMemcpyAsync((void*)d_rho, rho, b_rho, cudaMemcpyHostToDevice, b->stream));
    if (u) CK(cudaMemcpyAsync((void*)d_u, u, b_u, cudaMemcpyHostToDevice, b->stream));
    if (fneq) CK(cudaMemcpyAsync((void*)d_fneq, fneq, b_f, cudaMemcpyHostToDevice, b->stream));
    const int par = (int)(b->host_step & 1);
    CK(launch_init(b->store, b->d_dom + ctx->idx, I.h, d_rho, d_u, d_fneq, par, 1, b->stream));
    s = zero_fbox(b, I);
    if (s != LBM_OK) return s;
    s = refresh_alm(b);
    if (s != LBM_OK) return s;
    if (b->stream) CK(cudaStreamSynchronize(b->stream));
    else CK(cudaDeviceSynchronize());
    return LBM_OK;
}

lbm_status alm_add_turbine(lbm_ctx* ctx, const alm_turbine_desc* d, int* id_out)
{
    ENTER(ctx);
    if (!d) return fail(b, LBM_ERR_INVALID_ARG, "null turbine", false);
    if ((int)I.turb.size() >= kMaxTurbines) return fail(b, LBM_ERR_INVALID_ARG, "too many rotors", false);
    if (!turbine_counts_ok(d, kMaxElements) || I.h.n_el + d->n_blades * d->n_elements > kMaxElements)
        return fail(b, LBM_ERR_INVALID_ARG, "element count out of range", false);
    if (d->regularisation != ALM_REG_GAUSSIAN && d->regularisation != ALM_REG_ROMA)
        return fail(b, LBM_ERR_INVALID_ARG, "unknown regularisation", false);
    if (d->tip_loss != 0 && d->tip_loss != 1) return fail(b, LBM_ERR_INVALID_ARG, "tip_loss must be 0 or 1", false);
    const bool roma = d->regularisation == ALM_REG_ROMA;
    if (!roma && !(d->epsilon >= 0.5 && d->epsilon <= 5.0))
        return fail(b, LBM_ERR_INVALID_ARG, "epsilon must be in [0.5, 5]", false);
    if (!(d->radius > 0.0)) return fail(b, LBM_ERR_INVALID_ARG, "radius must be > 0", false);
    if (d->n_polar < 2 || !d->alpha || !d->cl || !d->cd) return fail(b, LBM_ERR_INVALID_ARG, "polar table missing", false);
    for (int i = 1; i < d->n_polar; ++i)
        if (!(d->alpha[i] > d->alpha[i - 1])) return fail(b, LBM_ERR_INVALID_ARG, "alpha must ascend", false);
    if (!turbine_values_finite(d)) return fail(b, LBM_ERR_INVALID_ARG, "non-finite rotor input", false);
    TurbineHost t;
    t.desc = *d;
    t.alpha.assign(d->alpha, d->alpha + d->n_polar);
    t.cl.assign(d->cl, d->cl + d->n_polar);
    t.cd.assign(d->cd, d->cd + d->n_polar);
    if (d->twist) t.twist.assign(d->twist, d->twist + d->n_elements);
    DevTurbine& B = t.dev;
    const double cy = std::cos(d->yaw), sy = std::sin(d->yaw);
    const double ea[3] = {cy, sy, 0.0}, e1[3] = {-sy, cy, 0.0}, e2[3] = {0.0, 0.0, 1.0};
    const int n[3] = {I.h.nx, I.h.ny, I.h.nz};
    const double cut = roma ? 1.5 : 3.0 * d->epsilon;
    for (int a = 0; a < 3; ++a) {
        B.hub[a] = (float)d->hub[a];
        B.e_axis[a] = (float)ea[a];
        B.e1[a] = (float)e1[a];
        B.e2[a] = (float)e2[a];
        const double ext = d->radius * std::sqrt(std::max(0.0, 1.0 - ea[a] * ea[a])) + cut + 1.0;
        B.lo[a] = (int)std::floor(d->hub[a] - ext);
        B.hi[a] = (int)std::ceil(d->hub[a] + ext);
        if (B.lo[a] < 1 || B.hi[a] > n[a] - 2)
            return fail(b, LBM_ERR_INVALID_ARG, "rotor force support must lie inside [1, n-2] on every axis", false);
    }
    B.radius = (float)d->radius;
    B.n_blades = d->n_blades;
    B.n_elements = d->n_elements;
    B.eps = roma ? 0.0f : (float)d->epsilon;
    B.inv_eps2 = roma ? 0.0f : (float)(1.0 / (d->epsilon * d->epsilon));
    B.cut = (float)cut;
    B.roma = roma ? 1 : 0;
    B.tip_loss = d->tip_loss;
    B.omega = d->omega;
    B.theta0 = d->theta0;
    B.pitch = (float)d->pitch;
    B.chord_root = (float)d->chord_root;
    B.chord_tip = (float)d->chord_tip;
    B.n_polar = d->n_polar;
    {
        // equally spaced angles (to 1e-6 of the spacing): direct segment index on the device
        const double da = (d->alpha[d->n_polar - 1] - d->alpha[0]) / (d->n_polar - 1);
        bool uni = da > 0.0;
        for (int i = 1; i < d->n_polar && uni; ++i)
            if (std::fabs((d->alpha[i] - d->alpha[i - 1]) - da) > 1e-6 * da) uni = false;
        B.polar_uniform = uni ? 1 : 0;
        B.polar_a0 = (float)d->alpha[0];
        B.polar_inv_da = uni ? (float)(1.0 / da) : 0.0f;
    }
    B.bnx = B.hi[0] - B.lo[0] + 1;
    B.bny = B.hi[1] - B.lo[1] + 1;
    B.bcells = (long long)B.bnx * B.bny * (B.hi[2] - B.lo[2] + 1);
    B.el_offset = I.h.n_el;
    std::vector<float> tab;
    for (double v : t.alpha) tab.push_back((float)v);
    for (double v : t.cl) tab.push_back((float)v);
    for (double v : t.cd) tab.push_back((float)v);
    for (double v : t.twist) tab.push_back((float)v);
    float* d_tab = (float*)dalloc(b, sizeof(float) * tab.size());
    float* d_fbox = (float*)dalloc(b, sizeof(float) * 3 * B.bcells);
    if (!d_tab || !d_fbox) return fail(b, LBM_ERR_OOM, "rotor table allocation failed");
    CK(cudaMemcpyAsync(d_tab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemsetAsync(d_fbox, 0, sizeof(float) * 3 * B.bcells, b->stream));
    B.alpha = d_tab;
    B.cl = d_tab + d->n_polar;
    B.cd = d_tab + 2 * d->n_polar;
    B.twist = d->twist ? d_tab + 3 * d->n_polar : nullptr;
    B.fbox = d_fbox;
    I.turb.push_back(std::move(t));
    I.h.n_turb = (int)I.turb.size();
    I.h.loads_sink = nullptr;  // a loads sink is sized for the rotors it was set with
    I.h.sink_len = 0;
    I.h.n_el += d->n_blades * d->n_elements;
    if (id_out) *id_out = (int)I.turb.size() - 1;
    b->dirty = true;
    lbm_status s = refresh_alm(b);
    if (s != LBM_OK) return s;
    if (b->stream) CK(cudaStreamSynchronize(b->stream));
    else CK(cudaDeviceSynchronize());
    return LBM_OK;
}

// Add the recorded event pairs to the running kernel time and free the pool.
lbm_status fold_events(Batch* b)
{
    if (b->ev_used == 0) return LBM_OK;
    CK(cudaEventSynchronize(b->ev[b->ev_used - 1]));
    for (size_t i = 0; i + 1 < b->ev_used; i += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, b->ev[i], b->ev[i + 1]));
        b->prof_ms += ms;
        b->prof_n += b->ev_launches[i / 2];
    }
    b->ev_used = 0;
    return LBM_OK;
}

// Steps per replay of the short and the long captured graph.
constexpr int kGraphSteps[2] = {2, 8};

// The captured graph of kGraphSteps[len] steps starting at parity p (source
// array f[p]); an even number of steps ends on the same parity.
lbm_status ensure_graph(Batch* b, int len, int p)
{
    if (b->gexec[len][p]) return LBM_OK;
    if (injected_fault("capture")) return fail(b, LBM_ERR_CUDA, "graph capture failed (injected: LBM_FAULT=capture)");
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    lbm_status s = LBM_OK;
    for (int i = 0; i < kGraphSteps[len] && s == LBM_OK; ++i) s = launch_one(b, p ^ (i & 1));
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (s != LBM_OK) return b->status;
    CK(e);
    e = cudaGraphInstantiate(&b->gexec[len][p], g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int n_steps)
{
    NvtxRange nvtx_("lbm_step");
    ENTER(ctx);
    if (n_steps < 0) return fail(b, LBM_ERR_INVALID_ARG, "n_steps < 0", false);
    if (const char* f = injected_fault("step")) {
        const long long at = *f == ':' ? std::atoll(f + 1) : 0;
        if (b->host_step <= at && at < b->host_step + n_steps)
            return fail(b, LBM_ERR_CUDA, "step " + std::to_string(at) + " failed (injected: LBM_FAULT=step:N)");
    }
    lbm_status s = sync_descriptors(b);
    if (s != LBM_OK) return s;
    long long left = n_steps;
    while (left > 0) {
        const int p = (int)(b->host_step & 1);
        // graphs (8 or 2 steps) cover no diagnostic step: those are single launches
        long long room = left;
        if (b->diag_every > 0) room = std::min(room, (b->diag_every - b->host_step % b->diag_every) % b->diag_every);
        const int len = room >= kGraphSteps[1] ? 1 : (room >= kGraphSteps[0] ? 0 : -1);
        const int k = (b->stream && len >= 0) ? kGraphSteps[len] : 1;
        if (k > 1) {
            s = ensure_graph(b, len, p);
            if (s != LBM_OK) return s;
        }
        if (b->profiling) {
            // events bracket each graph replay or single step, so timing does
            // not break up the replays
            if (b->ev_used + 2 > b->ev.size()) {
                if (b->ev.size() < 32768) {
                    cudaEvent_t e0, e1;
                    CK(cudaEventCreate(&e0));
                    CK(cudaEventCreate(&e1));
                    b->ev.push_back(e0);
                    b->ev.push_back(e1);
                    b->ev_launches.push_back(0);
                } else {
                    s = fold_events(b);
                    if (s != LBM_OK) return s;
                }
            }
            CK(cudaEventRecord(b->ev[b->ev_used], b->stream));
        }
        if (k > 1) {
            CK(cudaGraphLaunch(b->gexec[len][p], b->stream));
        } else {
            s = launch_one(b, p, b->diag_every > 0 && b->host_step % b->diag_every == 0);
            if (s != LBM_OK) return s;
        }
        if (b->profiling) {
            CK(cudaEventRecord(b->ev[b->ev_used + 1], b->stream));
            b->ev_launches[b->ev_used / 2] = k;
            b->ev_used += 2;
        }
        b->host_step += k;
        left -= k;
    }
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* ctx)
{
    ENTER(ctx);
    return check_device_errors(b);
}

lbm_status lbm_get_moments(lbm_ctx* ctx, double* rho, double* u)
{
    NvtxRange nvtx_("lbm_get_moments");
    ENTER(ctx);
    REQUIRE_EVEN_STEP();
    if (!rho || !u) return fail(b, LBM_ERR_INVALID_ARG, "null output", false);
    lbm_status s = sync_descriptors(b);
    if (s != LBM_OK) return s;
    const long long N = I.h.N;
    double* d = (double*)stage(b, sizeof(double) * 4 * N);
    if (!d) return fail(b, LBM_ERR_OOM, "moment buffer allocation failed");
    CK(launch_moments(b->store, b->d_dom + ctx->idx, I.h, (int)(b->host_step & 1), d, d + N, b->stream));
    CK(cudaMemcpyAsync(rho, d, sizeof(double) * N, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(u, d + N, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, b->stream));
    return check_device_errors(b);
}

lbm_status lbm_probe(lbm_ctx* ctx, const long long* cells, int n, double* rho, double* u)
{
    ENTER(ctx);
    REQUIRE_EVEN_STEP();
    if (n < 0 || (n > 0 && (!cells || !u))) return fail(b, LBM_ERR_INVALID_ARG, "bad probe arguments", false);
    if (n == 0) return LBM_OK;
    for (int k = 0; k < n; ++k)
        if (cells[k] < 0 || cells[k] >= I.h.N) return fail(b, LBM_ERR_INVALID_ARG, "probe cell out of range", false);
    lbm_status s = sync_descriptors(b);
    if (s != LBM_OK) return s;
    if (n > b->probe_cap) {
        dfree(b, b->d_probe);
        dfree(b, b->d_probe_out);
        b->probe_cap = 0;
        b->d_probe = (long long*)dalloc(b, sizeof(long long) * n);
        b->d_probe_out = (double*)dalloc(b, sizeof(double) * 4 * n);
        if (!b->d_probe || !b->d_probe_out) {
            dfree(b, b->d_probe);
            dfree(b, b->d_probe_out);
            b->d_probe = nullptr;
            b->d_probe_out = nullptr;
            return fail(b, LBM_ERR_OOM, "probe buffer allocation failed");
        }
        b->probe_cap = n;
    }
    CK(cudaMemcpyAsync(b->d_probe, cells, sizeof(long long) * n, cudaMemcpyHostToDevice, b->stream));
    CK(launch_probe(b->store, b->d_dom + ctx->idx, (int)(b->host_step & 1), b->d_probe, n, b->d_probe_out, b->stream));
    std::vector<double> out((size_t)4 * n);
    CK(cudaMemcpyAsync(out.data(), b->d_probe_out, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, b->stream));
    s = check_device_errors(b);
    if (s != LBM_OK) return s;
    for (int k = 0; k < n; ++k) {
        if (rho) rho[k] = out[4 * k];
        for (int a = 0; a < 3; ++a) u[3 * k + a] = out[4 * k + 1 + a];
    }
    return LBM_OK;
}

lbm_status lbm_get_pdfs(lbm_ctx* ctx, double* f)
{
    NvtxRange nvtx_("lbm_get_pdfs");
    ENTER(ctx);
    REQUIRE_EVEN_STEP();
    if (!f) return fail(b, LBM_ERR_INVALID_ARG, "null output", false);
    const long long N = I.h.N;
    const char* src = (const char*)I.h.f[b->host_step & 1];
    double* d = (double*)stage(b, sizeof(double) * N);
    if (!d) return fail(b, LBM_ERR_OOM, "staging allocation failed");
    // plane by plane: w_q + h on the device, then one copy to the caller's array
    for (int q = 0; q < 27; ++q) {
        CK(launch_plane_to_f64(b->store, src + (size_t)q * N * store_bytes(b->store), d, N, wqh(q), b->stream));
        CK(cudaMemcpyAsync(f + (size_t)q * N, d, sizeof(double) * N, cudaMemcpyDeviceToHost, b->stream));
    }
    return check_device_errors(b);
}

lbm_status lbm_set_pdfs(lbm_ctx* ctx, const double* f)
{
    NvtxRange nvtx_("lbm_set_pdfs");
    ENTER(ctx);
    REQUIRE_EVEN_STEP();
    if (!f) return fail(b, LBM_ERR_INVALID_ARG, "null input", false);
    const long long N = I.h.N;
    char* dst = (char*)I.h.f[b->host_step & 1];
    double* d = (double*)stage(b, sizeof(double) * N);
    if (!d) return fail(b, LBM_ERR_OOM, "staging allocation failed");
    for (int q = 0; q < 27; ++q) {
        CK(cudaMemcpyAsync(d, f + (size_t)q * N, sizeof(double) * N, cudaMemcpyHostToDevice, b->stream));
        CK(launch_plane_from_f64(b->store, d, dst + (size_t)q * N * store_bytes(b->store), N, wqh(q), b->stream));
    }
    lbm_status s = refresh_alm(b);
    if (s != LBM_OK) return s;
    return check_device_errors(b);
}

lbm_status alm_get_loads(lbm_ctx* ctx, int id, double* thrust, double* torque, float* elem_force, float* elem_pos)
{
    ENTER(ctx);
    if (id < 0 || id >= (int)I.turb.size()) return fail(b, LBM_ERR_INVALID_ARG, "bad rotor id", false);
    lbm_status s = check_device_errors(b);
    if (s != LBM_OK) return s;
    const int par = b->host_step > 0 ? (int)((b->host_step - 1) & 1) : 0;
    double L[2];
    CK(cudaMemcpy(L, I.h.loads[par] + 2 * id, sizeof L, cudaMemcpyDeviceToHost));
    if (thrust) *thrust = L[0];
    if (torque) *torque = L[1];
    const DevTurbine& B = I.turb[id].dev;
    const int ne = B.n_blades * B.n_elements;
    std::vector<float4> tmp(ne);
    if (elem_force) {
        CK(cudaMemcpy(tmp.data(), I.h.el_force[par] + B.el_offset, sizeof(float4) * ne, cudaMemcpyDeviceToHost));
        for (int e = 0; e < ne; ++e) {
            elem_force[3 * e] = tmp[e].x;
            elem_force[3 * e + 1] = tmp[e].y;
            elem_force[3 * e + 2] = tmp[e].z;
        }
    }
    if (elem_pos) {
        CK(cudaMemcpy(tmp.data(), I.h.el_pos[par] + B.el_offset, sizeof(float4) * ne, cudaMemcpyDeviceToHost));
        for (int e = 0; e < ne; ++e) {
            elem_pos[3 * e] = tmp[e].x;
            elem_pos[3 * e + 1] = tmp[e].y;
            elem_pos[3 * e + 2] = tmp[e].z;
        }
    }
    return LBM_OK;
}

lbm_status alm_get_loads_async(lbm_ctx* ctx, int id, double* thrust_torque)
{
    ENTER(ctx);
    if (id < 0 || id >= (int)I.turb.size()) return fail(b, LBM_ERR_INVALID_ARG, "bad rotor id", false);
    if (!thrust_torque) return fail(b, LBM_ERR_INVALID_ARG, "null output", false);
    // the slot of the last enqueued step; the next step's rotor launch, which
    // rewrites it, is ordered after this copy on the stream
    const int par = b->host_step > 0 ? (int)((b->host_step - 1) & 1) : 0;
    CK(cudaMemcpyAsync(thrust_torque, I.h.loads[par] + 2 * id, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                       b->stream));
    return LBM_OK;
}

lbm_status alm_set_loads_sink(lbm_ctx* ctx, double* host_ring, int ring_len)
{
    ENTER(ctx);
    if (!host_ring || ring_len <= 0) {
        I.h.loads_sink = nullptr;
        I.h.sink_len = 0;
    } else {
        void* dp = nullptr;
        if (cudaHostGetDevicePointer(&dp, host_ring, 0) != cudaSuccess) {
            cudaGetLastError();
            return fail(b, LBM_ERR_INVALID_ARG, "loads sink is not mapped page-locked host memory", false);
        }
        I.h.loads_sink = (double*)dp;
        I.h.sink_len = ring_len;
    }
    // the descriptor is read by the kernels: upload it before the next launch
    CK(cudaMemcpyAsync(b->d_dom + ctx->idx, &I.h, sizeof(DevDomain), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

lbm_status lbm_get_diagnostics(lbm_ctx* ctx, double mass_mom[4], long long* at_step)
{
    ENTER(ctx);
    if (!mass_mom) return fail(b, LBM_ERR_INVALID_ARG, "null output", false);
    lbm_status s = check_device_errors(b);
    if (s != LBM_OK) return s;
    double r[5];
    CK(cudaMemcpy(r, I.h.diag_res, sizeof r, cudaMemcpyDeviceToHost));
    for (int k = 0; k < 4; ++k) mass_mom[k] = r[k];
    if (at_step) *at_step = (long long)r[4];
    return LBM_OK;
}

lbm_status lbm_get_step(lbm_ctx* ctx, long long* step)
{
    ENTER(ctx);
    if (!step) return fail(b, LBM_ERR_INVALID_ARG, "null output", false);
    *step = b->host_step;
    return LBM_OK;
}

lbm_status lbm_set_step(lbm_ctx* ctx, long long step)
{
    ENTER(ctx);
    REQUIRE_EVEN_STEP();
    if (b->inplace && (step & 1))
        return fail(b, LBM_ERR_STATE, "in-place lattice: the step count must stay even", false);
    if (step < 0) return fail(b, LBM_ERR_INVALID_ARG, "step < 0", false);
    if ((step & 1) != (b->host_step & 1)) {
        // keep the live state in array f[step & 1]
        for (auto& In : b->inst) std::swap(In.h.f[0], In.h.f[1]);
        b->dirty = true;
    }
    b->host_step = step;
    CK(write_step_slot(b));
    lbm_status s = refresh_alm(b);
    if (s != LBM_OK) return s;
    return check_device_errors(b);
}

// ---------------------------------------------------------------- checkpoints

namespace {

// Header of a checkpoint blob; the sections follow in the order of
// state_sections().
struct StateHeader {
    char magic[8];
    int version;
    int nx, ny, nz, storage, collision, inplace;
    int bc[3];
    int n_turb, n_el;
    long long step;
    long long bcells[kMaxTurbines];
    unsigned long long bytes;  // whole blob
};
constexpr char kStateMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', 'E'};

struct Section {
    void* dev;
    size_t bytes;
};

// The device state one step reads and writes, beyond the descriptors: the
// PDFs of the current step, each rotor's lagged force box, the actuator-line
// element buffers and rotor loads of both step parities, the inlet ghost columns of
// both parities, and the last diagnostic sums.
std::vector<Section> state_sections(Batch* b, Instance& I)
{
    std::vector<Section> v;
    const DevDomain& h = I.h;
    v.push_back({h.f[b->host_step & 1], (size_t)h.N * 27 * store_bytes(b->store)});
    for (auto& t : I.turb) v.push_back({t.dev.fbox, sizeof(float) * 3 * (size_t)t.dev.bcells});
    if (h.n_el > 0)
        for (int p = 0; p < 2; ++p) {
            v.push_back({h.el_pos[p], sizeof(float4) * h.n_el});
            v.push_back({h.el_force[p], sizeof(float4) * h.n_el});
        }
    if (h.n_turb > 0)
        for (int p = 0; p < 2; ++p) v.push_back({h.loads[p], sizeof(double) * 2 * h.n_turb});
    if (h.inflow_ghost[0])
        for (int p = 0; p < 2; ++p) v.push_back({h.inflow_ghost[p], sizeof(float) * 9 * (size_t)h.ny * h.nz});
    if (h.outlet[0])
        for (int p = 0; p < 2; ++p) v.push_back({h.outlet[p], sizeof(float) * 9 * (size_t)h.ny * h.nz});
    v.push_back({h.diag_res, sizeof(double) * 5});
    return v;
}

StateHeader state_header(Batch* b, Instance& I)
{
    StateHeader H{};
    std::memcpy(H.magic, kStateMagic, 8);
    H.version = 1;
    H.nx = I.h.nx;
    H.ny = I.h.ny;
    H.nz = I.h.nz;
    H.storage = b->store;
    H.collision = b->coll;
    H.inplace = b->inplace;
    for (int a = 0; a < 3; ++a) H.bc[a] = I.h.bc[a];
    H.n_turb = I.h.n_turb;
    H.n_el = I.h.n_el;
    H.step = b->host_step;
    for (size_t t = 0; t < I.turb.size(); ++t) H.bcells[t] = I.turb[t].dev.bcells;
    size_t bytes = sizeof(StateHeader);
    for (auto& sec : state_sections(b, I)) bytes += sec.bytes;
    H.bytes = bytes;
    return H;
}

}  // namespace

lbm_status lbm_get_state_size(lbm_ctx* ctx, size_t* bytes)
{
    ENTER(ctx);
    if (!bytes) return fail(b, LBM_ERR_INVALID_ARG, "null output", false);
    *bytes = (size_t)state_header(b, I).bytes;
    return LBM_OK;
}

lbm_status lbm_get_state(lbm_ctx* ctx, void* buf, size_t bytes)
{
    NvtxRange nvtx_("lbm_get_state");
    ENTER(ctx);
    REQUIRE_EVEN_STEP();
    const StateHeader H = state_header(b, I);
    if (!buf || bytes < H.bytes) return fail(b, LBM_ERR_INVALID_ARG, "state buffer missing or too small", false);
    lbm_status s = sync_descriptors(b);
    if (s != LBM_OK) return s;
    std::memcpy(buf, &H, sizeof H);
    char* p = (char*)buf + sizeof H;
    for (auto& sec : state_sections(b, I)) {
        CK(cudaMemcpyAsync(p, sec.dev, sec.bytes, cudaMemcpyDeviceToHost, b->stream));
        p += sec.bytes;
    }
    return check_device_errors(b);
}

lbm_status lbm_set_state(lbm_ctx* ctx, const void* buf, size_t bytes)
{
    NvtxRange nvtx_("lbm_set_state");
    ENTER(ctx);
    REQUIRE_EVEN_STEP();
    if (!buf || bytes < sizeof(StateHeader)) return fail(b, LBM_ERR_INVALID_ARG, "state buffer missing or too small", false);
    StateHeader H;
    std::memcpy(&H, buf, sizeof H);
    const StateHeader mine = state_header(b, I);
    bool same = std::memcmp(H.magic, kStateMagic, 8) == 0 && H.version == 1 && H.nx == mine.nx && H.ny == mine.ny &&
                H.nz == mine.nz && H.storage == mine.storage && H.collision == mine.collision &&
                H.inplace == mine.inplace && H.n_turb == mine.n_turb && H.n_el == mine.n_el && H.bytes == mine.bytes;
    for (int a = 0; a < 3; ++a) same = same && H.bc[a] == mine.bc[a];
    for (int t = 0; t < kMaxTurbines; ++t) same = same && H.bcells[t] == mine.bcells[t];
    if (!same) return fail(b, LBM_ERR_INVALID_ARG, "state was taken from a lattice of another shape, storage or rotor set", false);
    if (bytes < H.bytes) return fail(b, LBM_ERR_INVALID_ARG, "state buffer too small", false);
    if (H.step < 0 || (b->inplace && (H.step & 1)))
        return fail(b, LBM_ERR_INVALID_ARG, "bad step in the state", false);
    lbm_status s = sync_descriptors(b);
    if (s != LBM_OK) return s;
    if ((H.step & 1) != (b->host_step & 1)) {
        // keep every lattice's live state in array f[step & 1]
        for (auto& In : b->inst) std::swap(In.h.f[0], In.h.f[1]);
        b->dirty = true;
    }
    b->host_step = H.step;
    s = sync_descriptors(b);
    if (s != LBM_OK) return s;
    const char* p = (const char*)buf + sizeof H;
    for (auto& sec : state_sections(b, I)) {
        CK(cudaMemcpyAsync(sec.dev, p, sec.bytes, cudaMemcpyHostToDevice, b->stream));
        p += sec.bytes;
    }
    CK(write_step_slot(b));
    return check_device_errors(b);
}

lbm_status lbm_set_wait_limit(lbm_ctx* ctx, long long cycles)
{
    ENTER(ctx);
    if (cycles < 0) return fail(b, LBM_ERR_INVALID_ARG, "wait limit < 0", false);
    b->wait_cycles = cycles;
    drop_graphs(b);  // the captured launches hold the old bound
    return LBM_OK;
}

// Staged rows need one-row tiles and every lattice's nx a multiple of the
// 16-byte chunk (4 FP32 or 8 16-bit values).
static bool staged_ok(Batch* b, int tile_y, int tile_z)
{
    if (tile_y != 1 || tile_z != 1) return false;
    const int chunk = b->store == STORE_FP32 ? 4 : 8;
    for (auto& I : b->inst)
        if (I.h.nx % chunk != 0) return false;
    return true;
}

lbm_status lbm_set_tile(lbm_ctx* ctx, int tile_x, int tile_y, int tile_z, int staged)
{
    ENTER(ctx);
    if (tile_x < 32 || tile_x % 32 != 0 || tile_y < 1 || tile_x * tile_y > 256 || tile_z < 1 || tile_z > 64)
        return fail(b, LBM_ERR_INVALID_ARG, "tile_x must be a multiple of 32, tile_x * tile_y <= 256, 1 <= tile_z <= 64",
                    false);
    if (staged < 0 || staged > 2) return fail(b, LBM_ERR_INVALID_ARG, "staged must be 0, 1 or 2", false);
    if (b->inplace && (tile_z != 1 || staged == 1))
        return fail(b, LBM_ERR_UNSUPPORTED, "the in-place scheme takes single-plane direct tiles only", false);
    if (staged == 1 && !staged_ok(b, tile_y, tile_z))
        return fail(b, LBM_ERR_INVALID_ARG, "staged rows need tile_y = tile_z = 1 and nx a multiple of 16 bytes", false);
    unsigned grid = 0;
    if (staged == 1) {
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int per_sm = staged_blocks_per_sm(b->coll, b->store, tile_x);
        if (per_sm < 1) return fail(b, LBM_ERR_INVALID_ARG, "staged tile does not fit on an SM", false);
        grid = (unsigned)(per_sm * sms);
    }
    b->tile_x = tile_x;
    b->tile_y = tile_y;
    b->tile_z = tile_z;
    b->staged = staged == 1 ? 1 : 0;
    b->single_cell = staged == 2 ? 1 : 0;
    b->staged_grid = grid;
    b->dirty = true;
    return sync_descriptors(b);
}

lbm_status lbm_get_tile(lbm_ctx* ctx, int* tile_x, int* tile_y, int* tile_z, int* staged)
{
    ENTER(ctx);
    if (tile_x) *tile_x = b->tile_x;
    if (tile_y) *tile_y = b->tile_y;
    if (tile_z) *tile_z = b->tile_z;
    if (staged) *staged = b->staged ? 1 : (b->single_cell ? 2 : 0);
    return LBM_OK;
}

namespace {

// Live state the tuner touches: the current PDF array and the rotor force boxes.
struct Snapshot {
    std::vector<void*> f;
    std::vector<float*> box;
};

lbm_status snapshot_take(Batch* b, Snapshot& S)
{
    const int cur = (int)(b->host_step & 1);
    for (auto& I : b->inst) {
        const size_t fb = (size_t)I.h.N * 27 * store_bytes(b->store);
        void* p = dalloc(b, fb);
        if (!p) return fail(b, LBM_ERR_OOM, "tuner snapshot allocation failed");
        CK(cudaMemcpyAsync(p, I.h.f[cur], fb, cudaMemcpyDeviceToDevice, b->stream));
        S.f.push_back(p);
        for (auto& t : I.turb) {
            float* q = (float*)dalloc(b, sizeof(float) * 3 * t.dev.bcells);
            if (!q) return fail(b, LBM_ERR_OOM, "tuner snapshot allocation failed");
            CK(cudaMemcpyAsync(q, t.dev.fbox, sizeof(float) * 3 * t.dev.bcells, cudaMemcpyDeviceToDevice, b->stream));
            S.box.push_back(q);
        }
    }
    return LBM_OK;
}

lbm_status snapshot_restore(Batch* b, const Snapshot& S, long long step)
{
    b->host_step = step;
    const int cur = (int)(step & 1);
    size_t k = 0;
    for (size_t i = 0; i < b->inst.size(); ++i) {
        Instance& I = b->inst[i];
        CK(cudaMemcpyAsync(I.h.f[cur], S.f[i], (size_t)I.h.N * 27 * store_bytes(b->store), cudaMemcpyDeviceToDevice,
                           b->stream));
        for (auto& t : I.turb) {
            CK(cudaMemcpyAsync(t.dev.fbox, S.box[k], sizeof(float) * 3 * t.dev.bcells, cudaMemcpyDeviceToDevice,
                               b->stream));
            ++k;
        }
    }
    CK(write_step_slot(b));
    return refresh_alm(b);
}

std::string tune_key(Batch* b)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    std::string k = "sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "/" + std::to_string(b->coll) +
                    "/" + std::to_string(b->store) + (b->inplace ? "/aa" : "");
    for (auto& I : b->inst) {
        k += "/" + std::to_string(I.h.nx) + "x" + std::to_string(I.h.ny) + "x" + std::to_string(I.h.nz);
        k += I.turb.empty() ? "" : "r" + std::to_string(I.turb.size());
    }
    return k;
}

}  // namespace

lbm_status lbm_autotune(lbm_ctx* ctx, int steps_per_candidate, const char* cache_path, int tile_out[4],
                        double* best_ms)
{
    NvtxRange nvtx_("lbm_autotune");
    ENTER(ctx);
    REQUIRE_EVEN_STEP();
    if (steps_per_candidate < 1) return fail(b, LBM_ERR_INVALID_ARG, "steps_per_candidate < 1", false);
    const std::string key = tune_key(b);
    if (cache_path) {
        if (FILE* fp = std::fopen(cache_path, "r")) {
            char kbuf[1024];
            int tx, ty, tz, st, hx = 0, hy = 0, hz = 0, hs = 0;
            double ms, hms = 0.0;
            bool hit = false;
            while (std::fscanf(fp, "%1023s %d %d %d %d %lf", kbuf, &tx, &ty, &tz, &st, &ms) == 6)
                if (key == kbuf) {
                    hit = true;
                    hx = tx;
                    hy = ty;
                    hz = tz;
                    hs = st;
                    hms = ms;
                }
            std::fclose(fp);
            if (hit) {
                if (tile_out) { tile_out[0] = hx; tile_out[1] = hy; tile_out[2] = hz; tile_out[3] = hs; }
                if (best_ms) *best_ms = hms;
                return lbm_set_tile(ctx, hx, hy, hz, hs);
            }
        }
    }
    // tile_x, tile_y, tile_z, staged
    // (staged 2: the single-plane shapes with one cell per thread, where the
    // bulk would otherwise take two)
    static const int cand[][4] = {{32, 4, 1, 0}, {32, 2, 1, 0}, {32, 8, 1, 0}, {64, 2, 1, 0}, {64, 1, 1, 0},
                                  {128, 1, 1, 0}, {64, 4, 1, 0}, {128, 2, 1, 0}, {32, 4, 2, 0}, {32, 4, 4, 0},
                                  {32, 2, 4, 0}, {32, 2, 8, 0}, {64, 2, 4, 0}, {32, 4, 8, 0}, {32, 4, 1, 2},
                                  {32, 8, 1, 2}, {64, 2, 1, 2}, {64, 1, 1, 2}, {64, 1, 1, 1}, {128, 1, 1, 1},
                                  {256, 1, 1, 1}};
    const long long step0 = b->host_step;
    const bool prof = b->profiling;
    Snapshot S;
    lbm_status s = sync_descriptors(b);
    if (s == LBM_OK) s = snapshot_take(b, S);
    int best = -1;
    double best_t = 1e300;
    for (int c = 0; s == LBM_OK && c < (int)(sizeof cand / sizeof cand[0]); ++c) {
        if (cand[c][3] == 1 && !staged_ok(b, cand[c][1], cand[c][2])) continue;
        if (cand[c][3] == 2 && !b->pairs_ok) continue;  // the same kernel as staged 0
        s = lbm_set_tile(ctx, cand[c][0], cand[c][1], cand[c][2], cand[c][3]);
        if (s == LBM_ERR_INVALID_ARG || s == LBM_ERR_UNSUPPORTED) {  // does not fit or not built: skip
            s = LBM_OK;
            continue;
        }
        if (s != LBM_OK) break;
        s = snapshot_restore(b, S, step0);
        if (s != LBM_OK) break;
        b->profiling = false;
        s = lbm_step(ctx, 3);
        if (s != LBM_OK) break;
        b->profiling = true;
        b->ev_used = 0;
        b->prof_ms = 0.0;
        b->prof_n = 0;
        s = lbm_step(ctx, steps_per_candidate);
        if (s != LBM_OK) break;
        double ms = 0.0;
        long long n = 0;
        s = lbm_get_kernel_time(ctx, &ms, &n);
        if (s == LBM_OK && ms < best_t) {
            best_t = ms;
            best = c;
        }
    }
    b->profiling = prof;
    b->ev_used = 0;
    b->prof_ms = 0.0;
    b->prof_n = 0;
    if (best >= 0 && s == LBM_OK) s = lbm_set_tile(ctx, cand[best][0], cand[best][1], cand[best][2], cand[best][3]);
    if (!S.f.empty() && s == LBM_OK) s = snapshot_restore(b, S, step0);
    for (void* p : S.f) dfree(b, p);
    for (float* p : S.box) dfree(b, p);
    if (s != LBM_OK) return s;
    if (best < 0) return fail(b, LBM_ERR_STATE, "no tile candidate ran");
    const int form = b->staged ? 1 : (b->single_cell ? 2 : 0);
    if (tile_out) { tile_out[0] = b->tile_x; tile_out[1] = b->tile_y; tile_out[2] = b->tile_z; tile_out[3] = form; }
    if (best_ms) *best_ms = best_t;
    if (cache_path)
        if (FILE* fp = std::fopen(cache_path, "a")) {
            std::fprintf(fp, "%s %d %d %d %d %.9g\n", key.c_str(), b->tile_x, b->tile_y, b->tile_z, form, best_t);
            std::fclose(fp);
        }
    return LBM_OK;
}

lbm_status lbm_set_profiling(lbm_ctx* ctx, int enable)
{
    ENTER(ctx);
    b->profiling = enable != 0;
    b->ev_used = 0;
    b->prof_ms = 0.0;
    b->prof_n = 0;
    return LBM_OK;
}

lbm_status lbm_get_kernel_time(lbm_ctx* ctx, double* mean_ms, long long* steps)
{
    ENTER(ctx);
    lbm_status s = fold_events(b);
    if (s != LBM_OK) return s;
    if (mean_ms) *mean_ms = b->prof_n ? b->prof_ms / (double)b->prof_n : 0.0;
    if (steps) *steps = b->prof_n;
    return LBM_OK;
}

lbm_status lbm_get_traffic_model(lbm_ctx* ctx, double* bytes_per_cell, long long* cells_per_step)
{
    ENTER(ctx);
    if (bytes_per_cell) *bytes_per_cell = 54.0 * (double)store_bytes(b->store);
    long long cells = 0;
    for (auto& In : b->inst) cells += In.h.N;
    if (cells_per_step) *cells_per_step = cells;
    return LBM_OK;
}

lbm_status lbm_get_launches_per_step(lbm_ctx* ctx, int* launches)
{
    ENTER(ctx);
    if (!launches) return fail(b, LBM_ERR_INVALID_ARG, "null output", false);
    lbm_status s = sync_descriptors(b);
    if (s != LBM_OK) return s;
    // the same split as launch_one
    // (with rotors: the rotor tiles and the actuator line)
    if (b->staged) *launches = 1 + (b->n_rotor > 0 ? 1 : 0);
    else if (b->inplace && !pair_tiles(b))
        *launches = (b->n_rotor > 0 ? 2 : 0) + (b->n_tiles > b->n_rotor ? 1 : 0);
    else
        *launches = (b->n_rotor > 0 ? 2 : 0) + (b->n_face > 0 ? 1 : 0) +
                    (b->n_tiles > b->n_rotor + b->n_face ? 1 : 0);
    return LBM_OK;
}

}  // extern "C"
