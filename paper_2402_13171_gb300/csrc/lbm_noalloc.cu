// Actuator-line evaluation that allocates no device memory (alm_eval_static in
// include/lbm_gb300.h).
//
// Some callers cannot allocate: a turbine-controller loop running under hard
// real-time limits, or code embedded in another framework that owns the
// device memory pool.  There, cudaMalloc/cudaFree are off limits: they may
// synchronise the whole device, take unbounded time, or be forbidden by the
// host framework.  This entry point runs the same actuator-line kernel as the
// lattice context (k_alm).  Its scratch (descriptors, polar table, per-corner
// samples, per-element loads and outputs) lives in one file-scope
// `static __device__` block that every GPU loading this library holds until
// the process exits.
//
// Rules of use:
//  - The first call on a device looks up the block's device address with
//    cudaGetSymbolAddress, with that device current.  Make that first call
//    before any stream capture.
//  - The rotor descriptor and polar table reach the block by copies from
//    pageable host memory (the call's own stack and a host vector), so the
//    call may wait for earlier work on its stream before it returns.
//  - All calls share the block and it keeps the last call's contents.  Calls
//    that overlap on the GPU (different streams, or host threads without
//    ordering) race on it; serialise them on one stream.
//  - Limits: at most kStaticMaxElements blade elements and kStaticMaxPolar
//    polar-table points per call; larger inputs are rejected with
//    LBM_ERR_INVALID_ARG before anything is enqueued.
#include "lbm_gb300.h"
#include "lbm_internal.h"

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <mutex>
#include <vector>

namespace lbmgb {

constexpr int kStaticMaxElements = 1024;
constexpr int kStaticMaxPolar = 8192;
constexpr int kMaxDevices = 64;

struct StaticScratch {
    DevDomain dom;
    DevTurbine turb;
    float4 el_pos[2][kStaticMaxElements];
    float4 el_force[2][kStaticMaxElements];
    double el_load[2 * kStaticMaxElements];
    double loads[2][2];
    float table[3 * kStaticMaxPolar + kStaticMaxElements];  // alpha, cl, cd, twist
    unsigned int err;
    unsigned int rotor_counter;
};

static __device__ __align__(256) StaticScratch g_alm_static;

// The actuator-line launch over the block's one lattice, of step `step`.
static AlmArgs alm_args_static(const DevDomain* d_dom, int n_el, long long step)
{
    AlmArgs a{};
    a.dom = d_dom;
    alm_blocks(a, &n_el, 1);
    a.step_slot = nullptr;
    a.step = step;
    a.array = 0;
    a.swapped = 0;
    return a;
}

namespace {
std::mutex g_mu;
StaticScratch* g_base[kMaxDevices] = {};

// Device address of the scratch block on the current device (looked up once).
cudaError_t scratch_base(StaticScratch** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_alm_static);
        if (e != cudaSuccess) return e;
        g_base[dev] = (StaticScratch*)p;
    }
    *out = g_base[dev];
    return cudaSuccess;
}
// Device address of member `off` bytes into the block (host arithmetic only).
template <typename M>
M* member(StaticScratch* base, size_t off)
{
    return reinterpret_cast<M*>(reinterpret_cast<char*>(base) + off);
}
}  // namespace

}  // namespace lbmgb

using namespace lbmgb;

extern "C" lbm_status alm_eval_static(const float* pdf_offsets, int nx, int ny, int nz, const double body_force[3],
                                      const alm_turbine_desc* d, long long step, float* elem_force, float* elem_pos,
                                      double* loads, void* cuda_stream)
{
    if (!pdf_offsets || !d || !elem_force || !loads || step < 0) return LBM_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 65535 || ny > 65535 || nz > 65535) return LBM_ERR_INVALID_ARG;
    const long long N = (long long)nx * ny * nz;
    if (27LL * N >= (1LL << 31)) return LBM_ERR_INVALID_ARG;
    if (!turbine_counts_ok(d, kStaticMaxElements)) return LBM_ERR_INVALID_ARG;
    const int n_el = d->n_blades * d->n_elements;
    if (d->n_polar < 2 || d->n_polar > kStaticMaxPolar || !d->alpha || !d->cl || !d->cd) return LBM_ERR_INVALID_ARG;
    if (d->regularisation != ALM_REG_GAUSSIAN && d->regularisation != ALM_REG_ROMA) return LBM_ERR_INVALID_ARG;
    if (d->tip_loss != 0 && d->tip_loss != 1) return LBM_ERR_INVALID_ARG;
    const bool roma = d->regularisation == ALM_REG_ROMA;
    if ((!roma && !(d->epsilon >= 0.5 && d->epsilon <= 5.0)) || !(d->radius > 0.0)) return LBM_ERR_INVALID_ARG;
    const double cut = roma ? 1.5 : 3.0 * d->epsilon;
    for (int i = 1; i < d->n_polar; ++i)
        if (!(d->alpha[i] > d->alpha[i - 1])) return LBM_ERR_INVALID_ARG;
    if (!turbine_values_finite(d)) return LBM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (body_force && !std::isfinite(body_force[a])) return LBM_ERR_INVALID_ARG;
    const double cy = std::cos(d->yaw), sy = std::sin(d->yaw);
    const double ea[3] = {cy, sy, 0.0}, e1[3] = {-sy, cy, 0.0}, e2[3] = {0.0, 0.0, 1.0};
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        // same support rule as alm_add_turbine: the sampled cells stay inside [1, n-2]
        const double ext = d->radius * std::sqrt(std::max(0.0, 1.0 - ea[a] * ea[a])) + cut + 1.0;
        if (std::floor(d->hub[a] - ext) < 1 || std::ceil(d->hub[a] + ext) > n[a] - 2) return LBM_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    StaticScratch* S = nullptr;
    if (scratch_base(&S) != cudaSuccess) return LBM_ERR_CUDA;

    // descriptors pointing into the static block; the blade force has no lagged
    // box force here (an empty box), only the body force
    DevTurbine B{};
    for (int a = 0; a < 3; ++a) {
        B.hub[a] = (float)d->hub[a];
        B.e_axis[a] = (float)ea[a];
        B.e1[a] = (float)e1[a];
        B.e2[a] = (float)e2[a];
        B.lo[a] = 1;
        B.hi[a] = 0;
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
        const double da = (d->alpha[d->n_polar - 1] - d->alpha[0]) / (d->n_polar - 1);
        bool uni = da > 0.0;
        for (int i = 1; i < d->n_polar && uni; ++i)
            if (std::fabs((d->alpha[i] - d->alpha[i - 1]) - da) > 1e-6 * da) uni = false;
        B.polar_uniform = uni ? 1 : 0;
        B.polar_a0 = (float)d->alpha[0];
        B.polar_inv_da = uni ? (float)(1.0 / da) : 0.0f;
    }
    float* tab = member<float>(S, offsetof(StaticScratch, table));
    DevTurbine* d_turb = member<DevTurbine>(S, offsetof(StaticScratch, turb));
    DevDomain* d_dom = member<DevDomain>(S, offsetof(StaticScratch, dom));
    float4* d_pos = member<float4>(S, offsetof(StaticScratch, el_pos));
    float4* d_force = member<float4>(S, offsetof(StaticScratch, el_force));
    double* d_loads = member<double>(S, offsetof(StaticScratch, loads));
    unsigned int* d_err = member<unsigned int>(S, offsetof(StaticScratch, err));
    B.alpha = tab;
    B.cl = tab + d->n_polar;
    B.cd = tab + 2 * d->n_polar;
    B.twist = d->twist ? tab + 3 * d->n_polar : nullptr;
    B.fbox = nullptr;
    B.bnx = B.bny = 0;
    B.bcells = 0;
    B.el_offset = 0;

    DevDomain D{};
    D.nx = nx;
    D.ny = ny;
    D.nz = nz;
    D.N = N;
    for (int a = 0; a < 3; ++a) D.body[a] = body_force ? (float)body_force[a] : 0.0f;
    D.f[0] = const_cast<float*>(pdf_offsets);
    D.f[1] = const_cast<float*>(pdf_offsets);
    D.n_turb = 1;
    D.turb = d_turb;
    for (int p = 0; p < 2; ++p) {
        D.el_pos[p] = d_pos + (size_t)p * kStaticMaxElements;
        D.el_force[p] = d_force + (size_t)p * kStaticMaxElements;
        D.loads[p] = d_loads + 2 * p;
    }
    D.el_load = member<double>(S, offsetof(StaticScratch, el_load));
    D.n_el = n_el;
    D.rotor_counter = member<unsigned int>(S, offsetof(StaticScratch, rotor_counter));
    D.err = d_err;

    std::vector<float> host_tab;
    host_tab.reserve(3 * d->n_polar + (d->twist ? d->n_elements : 0));
    for (int i = 0; i < d->n_polar; ++i) host_tab.push_back((float)d->alpha[i]);
    for (int i = 0; i < d->n_polar; ++i) host_tab.push_back((float)d->cl[i]);
    for (int i = 0; i < d->n_polar; ++i) host_tab.push_back((float)d->cd[i]);
    if (d->twist)
        for (int i = 0; i < d->n_elements; ++i) host_tab.push_back((float)d->twist[i]);

    const int par = (int)(step & 1);
    if (cudaMemcpyAsync(tab, host_tab.data(), sizeof(float) * host_tab.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_turb, &B, sizeof B, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_dom, &D, sizeof D, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(d_err, 0, sizeof(unsigned int), st) != cudaSuccess ||
        launch_alm(STORE_FP32, alm_args_static(d_dom, n_el, step), st, false) != cudaSuccess ||
        cudaMemcpy2DAsync(elem_force, 3 * sizeof(float), d_force + (size_t)par * kStaticMaxElements, sizeof(float4),
                          3 * sizeof(float), n_el, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(loads, d_loads + 2 * par, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (elem_pos &&
        cudaMemcpy2DAsync(elem_pos, 3 * sizeof(float), d_pos + (size_t)par * kStaticMaxElements, sizeof(float4),
                          3 * sizeof(float), n_el, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return LBM_ERR_CUDA;
    return LBM_OK;
}
