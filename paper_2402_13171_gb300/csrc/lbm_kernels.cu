// sm_103a kernels of the D3Q27 LBM + actuator line time step (arxiv 2402.13171).
//
// k_step: the fused pass of a time step over every cell of every lattice of a
// batch: pull streaming with boundary rules (Sec. 2.1, streaming step), force
// (body force + regularised blade forces, Sec. 2.2, gathered in the
// rotor box), collision (cumulant, Sec. 2.1 / Geier et al. 2015, or BGK with a
// Smagorinsky eddy viscosity), store.  PDFs live in HBM as offsets h = f - w
// in the storage type; all arithmetic is FP32.  A step with rotors is three
// launches: the tiles covering the rotor boxes (with the gather of the
// regularised blade forces); the actuator line of the next step (k_alm: blade
// kinematics of Algorithm 2, trilinear sampling, blade-element forces, FP64
// rotor loads), which waits on the device for the rotor tiles; and the rest of
// the lattice, which starts as soon as the rotor and actuator-line CTAs are
// resident and overlaps both.
#include "lbm_internal.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

namespace lbmgb {

// ------------------------------------------------------------------ lattice

__host__ __device__ constexpr int qcx(int q) { return q % 3 - 1; }
__host__ __device__ constexpr int qcy(int q) { return (q / 3) % 3 - 1; }
__host__ __device__ constexpr int qcz(int q) { return q / 9 - 1; }
// One-axis weights 2/3 and 1/6 as FP32 values whose sum w1(-1) + w1(0) + w1(1)
// is exactly 1 (2/3 rounded to nearest, 1/6 rounded down by 1e-8), so that the
// equilibrium parts added by the collision carry no one-signed mass or
// momentum error.
__host__ __device__ constexpr float w1(int c) { return c == 0 ? 0x1.555556p-1f : 0x1.555554p-3f; }
// w1(j) w1(k) for the x pass of the collision, rounded so that the nine values
// also sum to exactly 1 (corner 1/36, edge 1/9, centre 4/9, each within 4e-8)
__host__ __device__ constexpr float w2(int j, int k)
{
    return (j == 0 && k == 0) ? 0x1.c71c74p-2f : ((j == 0 || k == 0) ? 0x1.c71c7p-4f : 0x1.c71c7p-6f);
}
__host__ __device__ constexpr float wq(int q) { return w1(qcx(q)) * w1(qcy(q)) * w1(qcz(q)); }

// ------------------------------------------------------------------ storage

template <typename T> struct Io;
template <> struct Io<float> {
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float ldw(const float* p) { return *p; }
    static __device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
    static __device__ __forceinline__ float round(float v) { return v; }
};
// 16-bit loads ask L2 for the surrounding 256 bytes: a warp's 64-byte row
// segment is a quarter of that, and the rest is the same row of the next
// x-tiles, which the following CTAs load next (more bytes in flight per load
// instruction; DRAM traffic unchanged).
template <> struct Io<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p)
    {
        unsigned short v;
        asm("ld.global.nc.L2::256B.u16 %0, [%1];" : "=h"(v) : "l"(p));
        return __uint_as_float((unsigned)v << 16);
    }
    static __device__ __forceinline__ float ldcg(const __nv_bfloat16* p) { return __bfloat162float(__ldcg(p)); }
    static __device__ __forceinline__ float ldw(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};
template <> struct Io<__half> {
    static __device__ __forceinline__ float ld(const __half* p)
    {
        unsigned short v;
        asm("ld.global.nc.L2::256B.u16 %0, [%1];" : "=h"(v) : "l"(p));
        return __half2float(__ushort_as_half(v));
    }
    static __device__ __forceinline__ float ldcg(const __half* p) { return __half2float(__ldcg(p)); }
    static __device__ __forceinline__ float ldw(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ float round(float v) { return __half2float(__float2half_rn(v)); }
};

__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_float(__half v) { return __half2float(v); }

// ------------------------------------------------------------------ inflow

// splitmix64 (Steele, Lea, Flood 2014): k-th output of the generator started at `seed`.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long k)
{
    unsigned long long z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Inflow velocity of inlet column (y, z) at step n: mean profile u_ref * scale(z)
// plus, per component a, noise_amp * xi with xi = (r >> 11) 2^-53 * 2 - 1 from
// the splitmix64 output r for counter ((n nz + z) ny + y) 3 + a + 1.  In FP32
// only the top 24 of those 53 bits are kept (converted exactly), which moves xi
// by less than 2^-23, one FP32 ulp of xi.
__device__ __forceinline__ void inflow_velocity(const DevDomain* D, long long step, int y, int z, float u[3])
{
    const float scale = D->inflow_scale[z];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const unsigned long long counter =
            (((unsigned long long)step * (unsigned long long)D->nz + (unsigned long long)z) * (unsigned long long)D->ny +
             (unsigned long long)y) * 3ull + (unsigned long long)a;
        const unsigned long long r = splitmix64(D->seed, counter + 1ull);
        const float xi = (float)(unsigned)(r >> 40) * 0x1p-23f - 1.0f;
        u[a] = fmaf(D->noise_amp_f, xi, D->u_ref_f[a] * scale);
    }
}

// ------------------------------------------------------------------ equilibrium

// Per-axis factors of the product equilibrium, split as phi = w1 + dphi with
// dphi(0) = -u^2, dphi(+-1) = (u^2 +- u)/2 (index c+1).
__device__ __forceinline__ void axis_factors(float u, float ph[3], float dp[3])
{
    float u2 = u * u;
    dp[0] = 0.5f * (u2 - u);
    dp[1] = -u2;
    dp[2] = 0.5f * (u2 + u);
    ph[0] = w1(-1) + dp[0];
    ph[1] = w1(0) + dp[1];
    ph[2] = w1(1) + dp[2];
}

// out[q] = feq_q(1 + drho, u) - w_q, evaluated as a telescoped product so the
// result carries the absolute precision of the small terms.
__device__ __forceinline__ void feq_offsets(float drho, float ux, float uy, float uz, float out[27])
{
    float px[3], dx[3], py[3], dy[3], pz[3], dz[3];
    axis_factors(ux, px, dx);
    axis_factors(uy, py, dy);
    axis_factors(uz, pz, dz);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float P = py[j] * pz[k];
            const float Dd = dy[j] * pz[k] + w1(j - 1) * dz[k];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float A = fmaf(drho, px[i], dx[i]);
                out[k * 9 + j * 3 + i] = fmaf(A, P, w1(i - 1) * Dd);
            }
        }
    }
}

// Inlet ghost populations of column (y, z) for step `step`: the offsets
// feq_q(rho = 1, u_in) - w_q of the nine directions with c_x = +1 (the values
// the x = 0 cells pull across the inlet face from that column), written once
// per column and step instead of once per pulling cell and direction.
__device__ __forceinline__ void write_inlet_ghost(const DevDomain* D, long long step, int y, int z)
{
    float u[3];
    inflow_velocity(D, step, y, z, u);
    float* g = D->inflow_ghost[step & 1];
    const int plane = D->ny * D->nz, col = z * D->ny + y;
    // feq_q(1, u) - w_q = dphi_x phi_y phi_z + w1(c_x) (dphi_y phi_z + w1(c_y) dphi_z) for the
    // nine directions with c_x = +1, the axis factors formed once
    float px[3], dx[3], py[3], dy[3], pz[3], dz[3];
    axis_factors(u[0], px, dx);
    axis_factors(u[1], py, dy);
    axis_factors(u[2], pz, dz);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            g[(k * 3 + j) * plane + col] = dx[2] * py[j] * pz[k] + w1(1) * (dy[j] * pz[k] + w1(j - 1) * dz[k]);
}

// ------------------------------------------------------------------ moments

struct Moments {
    float drho, jx, jy, jz, Sxx, Syy, Szz, Sxy, Sxz, Syz;
};

// Raw moments of the offsets up to second order, summed axis by axis.
__device__ __forceinline__ Moments raw_moments(const float h[27])
{
    float m0[9], m1[9], m2[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const float a = h[3 * r], b = h[3 * r + 1], c = h[3 * r + 2];
        m2[r] = c + a;
        m0[r] = m2[r] + b;
        m1[r] = c - a;
    }
    float A00[3], A10[3], A20[3], A01[3], A11[3], A02[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int r0 = 3 * k, r1 = 3 * k + 1, r2 = 3 * k + 2;
        A02[k] = m0[r2] + m0[r0];
        A00[k] = A02[k] + m0[r1];
        A10[k] = m1[r0] + m1[r1] + m1[r2];
        A20[k] = m2[r0] + m2[r1] + m2[r2];
        A01[k] = m0[r2] - m0[r0];
        A11[k] = m1[r2] - m1[r0];
    }
    Moments M;
    M.Szz = A00[2] + A00[0];
    M.drho = M.Szz + A00[1];
    M.jx = A10[0] + A10[1] + A10[2];
    M.jy = A01[0] + A01[1] + A01[2];
    M.jz = A00[2] - A00[0];
    M.Sxx = A20[0] + A20[1] + A20[2];
    M.Syy = A02[0] + A02[1] + A02[2];
    M.Sxy = A11[0] + A11[1] + A11[2];
    M.Sxz = A10[2] - A10[0];
    M.Syz = A01[2] - A01[0];
    return M;
}

// ------------------------------------------------------------------ collisions

// One-dimensional map from central moments (k0, k1, k2) about u to the three
// populations at c = -1, 0, +1, taking h2 = k2/2:
//   f(-1) = dm k0 + (u - 1/2) k1 + h2,   f(+1) = dp k0 + (u + 1/2) k1 + h2,
//   f(0)  = k0 - f(-1) - f(+1)           (the map preserves the zeroth moment)
// with dm = (u^2 - u)/2 and dp = (u^2 + u)/2.  (dm, -u^2, dp) is also the
// deviation dphi of the equilibrium factor phi(c) = w1(c) + dphi(c), the map
// applied to the equilibrium central moments (1, 0, 1/3).
struct Axis {
    float dm, dp, u2, bm, bp;
};

__device__ __forceinline__ Axis axis_of(float u)
{
    Axis a;
    a.u2 = u * u;
    a.dm = 0.5f * (a.u2 - u);
    a.dp = 0.5f * (a.u2 + u);
    a.bm = u - 0.5f;
    a.bp = u + 0.5f;
    return a;
}

__device__ __forceinline__ float dphi(const Axis& a, int c) { return c < 0 ? a.dm : (c > 0 ? a.dp : -a.u2); }

// the map for general (k0, k1, h2) and for the zero patterns of the collided moments
__device__ __forceinline__ void inv_full(const Axis& a, float k0, float k1, float h2, float& fm, float& f0, float& fp)
{
    fm = fmaf(a.dm, k0, fmaf(a.bm, k1, h2));
    fp = fmaf(a.dp, k0, fmaf(a.bp, k1, h2));
    f0 = k0 - fm - fp;
}
__device__ __forceinline__ void inv_k1h2(const Axis& a, float k1, float h2, float& fm, float& f0, float& fp)
{
    fm = fmaf(a.bm, k1, h2);
    fp = fmaf(a.bp, k1, h2);
    f0 = -fm - fp;
}
__device__ __forceinline__ void inv_k0k1(const Axis& a, float k0, float k1, float& fm, float& f0, float& fp)
{
    fm = fmaf(a.dm, k0, a.bm * k1);
    fp = fmaf(a.dp, k0, a.bp * k1);
    f0 = k0 - fm - fp;
}
__device__ __forceinline__ void inv_k0h2(const Axis& a, float k0, float h2, float& fm, float& f0, float& fp)
{
    fm = fmaf(a.dm, k0, h2);
    fp = fmaf(a.dp, k0, h2);
    f0 = k0 - fm - fp;
}
__device__ __forceinline__ void inv_k1(const Axis& a, float k1, float& fm, float& f0, float& fp)
{
    fm = a.bm * k1;
    fp = a.bp * k1;
    f0 = -fm - fp;
}

// ------------------------------------------------------------------ packed FP32 pairs

// The f32x2 forms of add, sub, mul and fma (sm_100 and later): one instruction
// on two FP32 lanes, each rounded exactly as the scalar instruction, so a
// paired evaluation gives the scalar evaluation's bits in half the issue slots.
#define LBM_F32X2(op)                                                                                        \
    "{\n .reg .b64 x_, y_, r_;\n mov.b64 x_, {%2, %3};\n mov.b64 y_, {%4, %5};\n " op                    \
    " r_, x_, y_;\n mov.b64 {%0, %1}, r_;\n}"
__device__ __forceinline__ float2 add2(float2 x, float2 y)
{
    float2 r;
    asm(LBM_F32X2("add.rn.f32x2") : "=f"(r.x), "=f"(r.y) : "f"(x.x), "f"(x.y), "f"(y.x), "f"(y.y));
    return r;
}
__device__ __forceinline__ float2 sub2(float2 x, float2 y)
{
    float2 r;
    asm(LBM_F32X2("sub.rn.f32x2") : "=f"(r.x), "=f"(r.y) : "f"(x.x), "f"(x.y), "f"(y.x), "f"(y.y));
    return r;
}
__device__ __forceinline__ float2 mul2(float2 x, float2 y)
{
    float2 r;
    asm(LBM_F32X2("mul.rn.f32x2") : "=f"(r.x), "=f"(r.y) : "f"(x.x), "f"(x.y), "f"(y.x), "f"(y.y));
    return r;
}
#undef LBM_F32X2
__device__ __forceinline__ float2 fma2(float2 x, float2 y, float2 z)
{
    float2 r;
    asm("{\n .reg .b64 x_, y_, z_, r_;\n mov.b64 x_, {%2, %3};\n mov.b64 y_, {%4, %5};\n mov.b64 z_, {%6, %7};\n"
        " fma.rn.f32x2 r_, x_, y_, z_;\n mov.b64 {%0, %1}, r_;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(x.x), "f"(x.y), "f"(y.x), "f"(y.y), "f"(z.x), "f"(z.y));
    return r;
}
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

// ------------------------------------------------------------------ lane types of the collision

// The cumulant collision is written once for two lane types: float (one cell)
// and float2 (the cells x and x + 1 of a row, one per lane).  Every operation
// is explicit and correctly rounded, with no contraction of a product into a
// sum left to the compiler, and the f32x2 instructions round each lane exactly
// as the scalar instruction, so a pair of cells evaluated on float2 gives bit
// for bit the values of the two cells evaluated one at a time on float.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return add2(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return sub2(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return mul2(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return fma2(a, b, c); }
__device__ __forceinline__ float2 vneg(float2 a) { return mul2(a, bc2(-1.0f)); }  // exact, signed zeros included
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(__frcp_rn(a.x), __frcp_rn(a.y)); }
template <class V> __device__ __forceinline__ V vc(float c);
template <> __device__ __forceinline__ float vc<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 vc<float2>(float c) { return bc2(c); }

// The values of the levels c_z = -1 (lo) and c_z = +1 (hi) of a lane type,
// carried together through the collision's passes: a float2 for one cell, two
// float2 (each over the two cells) for a pair of cells.
struct float2x2 {
    float2 lo, hi;
};
template <class V> struct ZPair;
template <> struct ZPair<float> { using T = float2; };
template <> struct ZPair<float2> { using T = float2x2; };
__device__ __forceinline__ float2 zmk(float lo, float hi) { return make_float2(lo, hi); }
__device__ __forceinline__ float2x2 zmk(float2 lo, float2 hi) { return {lo, hi}; }
__device__ __forceinline__ float zlo(float2 p) { return p.x; }
__device__ __forceinline__ float zhi(float2 p) { return p.y; }
__device__ __forceinline__ float2 zlo(const float2x2& p) { return p.lo; }
__device__ __forceinline__ float2 zhi(const float2x2& p) { return p.hi; }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return add2(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return sub2(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return mul2(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return fma2(a, b, c); }
__device__ __forceinline__ float2x2 padd(const float2x2& a, const float2x2& b) { return {add2(a.lo, b.lo), add2(a.hi, b.hi)}; }
__device__ __forceinline__ float2x2 psub(const float2x2& a, const float2x2& b) { return {sub2(a.lo, b.lo), sub2(a.hi, b.hi)}; }
__device__ __forceinline__ float2x2 pmul(const float2x2& a, const float2x2& b) { return {mul2(a.lo, b.lo), mul2(a.hi, b.hi)}; }
__device__ __forceinline__ float2x2 pfma(const float2x2& a, const float2x2& b, const float2x2& c)
{
    return {fma2(a.lo, b.lo, c.lo), fma2(a.hi, b.hi, c.hi)};
}
template <class V> __device__ __forceinline__ typename ZPair<V>::T pbc(V v) { return zmk(v, v); }

template <class V>
struct MomentsV {
    V drho, jx, jy, jz, Sxx, Syy, Szz, Sxy, Sxz, Syz;
};

// Raw moments as raw_moments computes them (same operations, same order), with
// the populations of the planes c_z = -1 and c_z = +1 carried as pairs:
// hp[3j + i] = (h[3j + i], h[18 + 3j + i]), hs[3j + i] = h[9 + 3j + i].
template <class V>
__device__ __forceinline__ MomentsV<V> raw_moments_paired(const typename ZPair<V>::T hp[9], const V hs[9])
{
    using P = typename ZPair<V>::T;
    P m0p[3], m1p[3], m2p[3];
    V m0s[3], m1s[3], m2s[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        m2p[j] = padd(hp[3 * j + 2], hp[3 * j]);
        m0p[j] = padd(m2p[j], hp[3 * j + 1]);
        m1p[j] = psub(hp[3 * j + 2], hp[3 * j]);
        m2s[j] = vadd(hs[3 * j + 2], hs[3 * j]);
        m0s[j] = vadd(m2s[j], hs[3 * j + 1]);
        m1s[j] = vsub(hs[3 * j + 2], hs[3 * j]);
    }
    // per z level k: pairs hold levels 0 and 2, the single values level 1
    const P A02p = padd(m0p[2], m0p[0]);
    const P A00p = padd(A02p, m0p[1]);
    const P A10p = padd(padd(m1p[0], m1p[1]), m1p[2]);
    const P A20p = padd(padd(m2p[0], m2p[1]), m2p[2]);
    const P A01p = psub(m0p[2], m0p[0]);
    const P A11p = psub(m1p[2], m1p[0]);
    const V A02s = vadd(m0s[2], m0s[0]);
    const V A00s = vadd(A02s, m0s[1]);
    const V A10s = vadd(vadd(m1s[0], m1s[1]), m1s[2]);
    const V A20s = vadd(vadd(m2s[0], m2s[1]), m2s[2]);
    const V A01s = vsub(m0s[2], m0s[0]);
    const V A11s = vsub(m1s[2], m1s[0]);
    MomentsV<V> M;
    M.Szz = vadd(zhi(A00p), zlo(A00p));
    M.drho = vadd(M.Szz, A00s);
    M.jx = vadd(vadd(zlo(A10p), A10s), zhi(A10p));
    M.jy = vadd(vadd(zlo(A01p), A01s), zhi(A01p));
    M.jz = vsub(zhi(A00p), zlo(A00p));
    M.Sxx = vadd(vadd(zlo(A20p), A20s), zhi(A20p));
    M.Syy = vadd(vadd(zlo(A02p), A02s), zhi(A02p));
    M.Sxy = vadd(vadd(zlo(A11p), A11s), zhi(A11p));
    M.Sxz = vsub(zhi(A10p), zlo(A10p));
    M.Syz = vsub(zhi(A01p), zlo(A01p));
    return M;
}

// The one-dimensional map of the passes (see Axis) on a lane type.
template <class V>
struct AxisV {
    V dm, dp, u2, bm, bp;
};
template <class V>
__device__ __forceinline__ AxisV<V> axis_of_v(V u)
{
    AxisV<V> a;
    a.u2 = vmul(u, u);
    a.dm = vmul(vc<V>(0.5f), vsub(a.u2, u));
    a.dp = vmul(vc<V>(0.5f), vadd(a.u2, u));
    a.bm = vsub(u, vc<V>(0.5f));
    a.bp = vadd(u, vc<V>(0.5f));
    return a;
}
template <class V>
__device__ __forceinline__ void inv_full_v(const AxisV<V>& a, V k0, V k1, V h2, V& fm, V& f0, V& fp)
{
    fm = vfma(a.dm, k0, vfma(a.bm, k1, h2));
    fp = vfma(a.dp, k0, vfma(a.bp, k1, h2));
    f0 = vsub(vsub(k0, fm), fp);
}

// Cumulant collision with shear rate omega, bulk and all higher-order rates 1
// (all cumulants above second order relax to zero, so post-collision central
// moments of order 4 and 6 are the Gaussian products of the second-order ones,
// orders 3 and 5 vanish), forcing by the velocity shift (first central moments
// -F/2 -> +F/2).
//
// The post-collision central moments are K = rho e0 (x) e0 (x) e0 + Delta with
// e0 = (1, 0, 1/3) the per-axis equilibrium moments and Delta the 16 nonzero
// collided deviations.  The populations f* = L_x L_y L_z K are formed pass by
// pass as offsets from the weights: since L_a e0 = w1 + dphi_a, each pass
// carries only the deviation, adding the equilibrium part that it owns
// (z: e0_a e0_b (dphi_z + drho phi_z), y: e0_a w1 dphi_y, x: w1 w1 dphi_x), so
// no large term is ever subtracted (in the y and x passes the part enters the
// pass input as the moments (0, u, -u^2), which the map takes to dphi).
// Second-order indices are held halved
// (moment (a, b, c) scaled by 2^-(number of indices equal to 2)), so that every
// pass receives h2 = k2/2 directly.
//
// The values of the z levels c_z = -1 and +1 travel as pairs through all
// three passes: the z pass produces them together (its f(-1), f(+1)), and the
// y and x passes treat the two levels alike (their weights are even in c_z), so
// for one cell those passes run on f32x2 instructions for two thirds of their
// columns.  V = float2 evaluates two cells on f32x2 instructions throughout.
template <class V>
__device__ __forceinline__ void collide_cumulant_v(V h[27], V Fx, V Fy, V Fz, float omega, V& drho_o, V& jx_o,
                                                   V& jy_o, V& jz_o)
{
    using P = typename ZPair<V>::T;
    P hp[9];
    V hs[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        hp[r] = zmk(h[r], h[18 + r]);
        hs[r] = h[9 + r];
    }
    const MomentsV<V> M = raw_moments_paired<V>(hp, hs);
    const V rho = vadd(vc<V>(1.0f), M.drho);
    // correctly rounded: the equilibrium momentum rho (j + F/2)/rho must not
    // carry a one-signed reciprocal error, or the lattice momentum drifts
    const V inv = vrcp(rho);
    const V hFx = vmul(vc<V>(0.5f), Fx), hFy = vmul(vc<V>(0.5f), Fy), hFz = vmul(vc<V>(0.5f), Fz);
    const V ux = vmul(vadd(M.jx, hFx), inv);
    const V uy = vmul(vadd(M.jy, hFy), inv);
    const V uz = vmul(vadd(M.jz, hFz), inv);
    const float third = 1.0f / 3.0f;
    // second central moments minus rho/3 delta, using rho u = j + F/2:
    //   S_ab - rho u_a u_b + (u_a F_b + u_b F_a)/2 = S_ab - j_a u_b + u_a F_b/2
    const V axx = vfma(ux, vsub(hFx, M.jx), vfma(M.drho, vc<V>(-third), M.Sxx));
    const V ayy = vfma(uy, vsub(hFy, M.jy), vfma(M.drho, vc<V>(-third), M.Syy));
    const V azz = vfma(uz, vsub(hFz, M.jz), vfma(M.drho, vc<V>(-third), M.Szz));
    const V njx = vneg(M.jx), njy = vneg(M.jy);
    const V axy = vfma(njx, uy, vfma(ux, hFy, M.Sxy));
    const V axz = vfma(njx, uz, vfma(ux, hFz, M.Sxz));
    const V ayz = vfma(njy, uz, vfma(uy, hFz, M.Syz));
    const V om1 = vc<V>(1.0f - omega);
    const V tr = vadd(vadd(axx, ayy), azz);
    const V bxx = vmul(om1, vfma(tr, vc<V>(-third), axx));
    const V byy = vmul(om1, vfma(tr, vc<V>(-third), ayy));
    const V bzz = vmul(om1, vfma(tr, vc<V>(-third), azz));
    const V bxy = vmul(om1, axy), bxz = vmul(om1, axz), byz = vmul(om1, ayz);
    const V inv2 = vmul(vc<V>(0.5f), inv), inv4 = vmul(vc<V>(0.25f), inv);
    const V b2xy = vadd(bxy, bxy), b2xz = vadd(bxz, bxz), b2yz = vadd(byz, byz);
    // collided deviations in the halved basis: orders 4 and 6 are the Gaussian
    // (Isserlis) products of the collided second-order moments minus those of
    // the equilibrium, expanded so that no equilibrium-sized term cancels
    const V d200 = vmul(vc<V>(0.5f), bxx), d020 = vmul(vc<V>(0.5f), byy), d002 = vmul(vc<V>(0.5f), bzz);
    const V c12 = vc<V>(1.0f / 12.0f), c6 = vc<V>(1.0f / 6.0f);
    const V d220 = vfma(vadd(bxx, byy), c12, vmul(vfma(bxx, byy, vmul(bxy, b2xy)), inv4));
    const V d202 = vfma(vadd(bxx, bzz), c12, vmul(vfma(bxx, bzz, vmul(bxz, b2xz)), inv4));
    const V d022 = vfma(vadd(byy, bzz), c12, vmul(vfma(byy, bzz, vmul(byz, b2yz)), inv4));
    const V d211 = vfma(byz, c6, vmul(vfma(bxx, byz, vmul(bxy, b2xz)), inv2));
    const V d121 = vfma(bxz, c6, vmul(vfma(byy, bxz, vmul(bxy, b2yz)), inv2));
    const V d112 = vfma(bxy, c6, vmul(vfma(bzz, bxy, vmul(bxz, b2yz)), inv2));
    V d222;
    {
        // g = s_xx s_yy s_zz-type product of (1/3 + s) minus 1/27, plus the
        // off-diagonal pairings, with s = b / rho
        const V sxx = vmul(bxx, inv), syy = vmul(byy, inv), szz = vmul(bzz, inv);
        const V sxy = vmul(bxy, inv), sxz = vmul(bxz, inv), syz = vmul(byz, inv);
        const V p = vadd(sxx, syy), q = vmul(sxx, syy);
        const V t = vc<V>(third);
        const V diag = vfma(vadd(p, szz), vc<V>(1.0f / 9.0f), vfma(vfma(szz, p, q), t, vmul(q, szz)));
        const V pair = vfma(vadd(t, sxx), vmul(syz, syz),
                            vfma(vadd(t, syy), vmul(sxz, sxz), vmul(vadd(t, szz), vmul(sxy, sxy))));
        const V g = vfma(vc<V>(2.0f), pair, vfma(vmul(vc<V>(8.0f), sxy), vmul(sxz, syz), diag));
        d222 = vmul(vmul(vc<V>(0.125f), rho), g);
    }
    const AxisV<V> X = axis_of_v(ux), Y = axis_of_v(uy), Z = axis_of_v(uz);
    // z pass over the columns (a, b): the pair (f(-1), f(+1)) = Gp[3b + a] and
    // f(0) = Gs[3b + a]; the map's coefficients enter as pairs (dm, dp), (bm, bp)
    const P zd = zmk(Z.dm, Z.dp), zb = zmk(Z.bm, Z.bp);
    P Gp[9];
    V Gs[9];
    auto z_k1h2 = [&](int c, V k1, V h2) {
        Gp[c] = pfma(zb, pbc(k1), pbc(h2));
        Gs[c] = vsub(vneg(zlo(Gp[c])), zhi(Gp[c]));
    };
    auto z_k0k1 = [&](int c, V k0, V k1) {
        Gp[c] = pfma(zd, pbc(k0), pmul(zb, pbc(k1)));
        Gs[c] = vsub(vsub(k0, zlo(Gp[c])), zhi(Gp[c]));
    };
    auto z_k0h2 = [&](int c, V k0, V h2) {
        Gp[c] = pfma(zd, pbc(k0), pbc(h2));
        Gs[c] = vsub(vsub(k0, zlo(Gp[c])), zhi(Gp[c]));
    };
    auto z_k1 = [&](int c, V k1) {
        Gp[c] = pmul(zb, pbc(k1));
        Gs[c] = vsub(vneg(zlo(Gp[c])), zhi(Gp[c]));
    };
    z_k1h2(0, hFz, d002);
    z_k0k1(1, hFx, bxz);
    z_k0h2(2, d200, d202);
    z_k0k1(3, hFy, byz);
    z_k0h2(4, bxy, d112);
    z_k1(5, d211);
    z_k0h2(6, d020, d022);
    z_k1(7, d121);
    z_k0h2(8, d220, d222);
    {
        // equilibrium part of the z pass: rho phi_z - w1 on the columns (0, 0),
        // (2, 0), (0, 2), (2, 2) with the weights 1, 1/6, 1/6, 1/36
        const P gzp = pfma(pbc(M.drho), padd(pbc(vc<V>(w1(1))), zd), zd);  // w1(-1) = w1(+1)
        Gp[0] = padd(Gp[0], gzp);
        Gp[2] = pfma(pbc(vc<V>(1.0f / 6.0f)), gzp, Gp[2]);
        Gp[6] = pfma(pbc(vc<V>(1.0f / 6.0f)), gzp, Gp[6]);
        Gp[8] = pfma(pbc(vc<V>(1.0f / 36.0f)), gzp, Gp[8]);
        const V dz = vneg(Z.u2);
        const V gz = vfma(M.drho, vadd(vc<V>(w1(0)), dz), dz);
        Gs[0] = vadd(Gs[0], gz);
        Gs[2] = vfma(vc<V>(1.0f / 6.0f), gz, Gs[2]);
        Gs[6] = vfma(vc<V>(1.0f / 6.0f), gz, Gs[6]);
        Gs[8] = vfma(vc<V>(1.0f / 36.0f), gz, Gs[8]);
    }
    // y pass over the columns (a, k); the equilibrium part e0_a w1 dphi_y enters
    // as the moments (0, u_y, -u_y^2), which the map takes to dphi_y
    const P ydm = pbc(Y.dm), ydp = pbc(Y.dp), ybm = pbc(Y.bm), ybp = pbc(Y.bp);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        P k1p = Gp[3 + a], h2p = Gp[6 + a];
        V k1s = Gs[3 + a], h2s = Gs[6 + a];
        if (a != 1) {
            const float ea = a == 0 ? 1.0f : 1.0f / 6.0f;
            const float ep = ea * w1(1), es = ea * w1(0);  // w1(-1) = w1(+1)
            k1p = pfma(pbc(vc<V>(ep)), pbc(uy), k1p);
            h2p = pfma(pbc(vc<V>(-0.5f * ep)), pbc(Y.u2), h2p);
            k1s = vfma(vc<V>(es), uy, k1s);
            h2s = vfma(vc<V>(-0.5f * es), Y.u2, h2s);
        }
        const P k0p = Gp[a];
        const P fm = pfma(ydm, k0p, pfma(ybm, k1p, h2p));
        const P fp = pfma(ydp, k0p, pfma(ybp, k1p, h2p));
        Gp[a] = fm;
        Gp[3 + a] = psub(psub(k0p, fm), fp);
        Gp[6 + a] = fp;
        inv_full_v(Y, Gs[a], k1s, h2s, Gs[a], Gs[3 + a], Gs[6 + a]);
    }
    // x pass over the rows (j, k), with w1 w1 dphi_x entered the same way
    const P xdm = pbc(X.dm), xdp = pbc(X.dp), xbm = pbc(X.bm), xbp = pbc(X.bp);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float ep = w2(j - 1, 1), es = w2(j - 1, 0);  // w2(j, -1) = w2(j, +1)
        const P k1p = pfma(pbc(vc<V>(ep)), pbc(ux), Gp[3 * j + 1]);
        const P h2p = pfma(pbc(vc<V>(-0.5f * ep)), pbc(X.u2), Gp[3 * j + 2]);
        const P k0p = Gp[3 * j];
        const P fm = pfma(xdm, k0p, pfma(xbm, k1p, h2p));
        const P fp = pfma(xdp, k0p, pfma(xbp, k1p, h2p));
        const P f0 = psub(psub(k0p, fm), fp);
        h[3 * j] = zlo(fm);
        h[3 * j + 1] = zlo(f0);
        h[3 * j + 2] = zlo(fp);
        h[18 + 3 * j] = zhi(fm);
        h[18 + 3 * j + 1] = zhi(f0);
        h[18 + 3 * j + 2] = zhi(fp);
        const V k1s = vfma(vc<V>(es), ux, Gs[3 * j + 1]), h2s = vfma(vc<V>(-0.5f * es), X.u2, Gs[3 * j + 2]);
        inv_full_v(X, Gs[3 * j], k1s, h2s, h[9 + 3 * j], h[9 + 3 * j + 1], h[9 + 3 * j + 2]);
    }
    drho_o = M.drho;
    jx_o = vadd(M.jx, Fx);
    jy_o = vadd(M.jy, Fy);
    jz_o = vadd(M.jz, Fz);
}

// One cell (the form every kernel but the paired bulk kernel uses).
__device__ __forceinline__ void collide_cumulant(float h[27], float Fx, float Fy, float Fz, float omega, float& drho_o,
                                                 float& jx_o, float& jy_o, float& jz_o)
{
    collide_cumulant_v<float>(h, Fx, Fy, Fz, omega, drho_o, jx_o, jy_o, jz_o);
}

// BGK toward the polynomial equilibrium with a Smagorinsky eddy viscosity
// (tau = (tau0 + sqrt(tau0^2 + 18 sqrt(2) C^2 |Pi|/rho))/2, Pi the
// force-corrected non-equilibrium momentum flux) and the Guo source
// (1 - omega/2) w [3(c - u) + 9 (c.u) c].F, on a lane type like the cumulant
// collision.  The raw moments take the f32x2 pairs of the cumulant collision;
// everything after them runs, on a pair of cells, as the one-cell scalar
// instructions lane by lane (sadd, smul, ... below), so the two forms agree bit
// for bit by construction (the f32x2 form of this part did not, in a fraction of
// the cells, although each f32x2 instruction rounds as its scalar one).
__device__ __forceinline__ float sadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float ssub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float smul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float sfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float sneg(float a) { return -a; }
__device__ __forceinline__ float2 sadd(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 ssub(float2 a, float2 b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
__device__ __forceinline__ float2 smul(float2 a, float2 b) { return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
__device__ __forceinline__ float2 sfma(float2 a, float2 b, float2 c)
{
    return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 sneg(float2 a) { return make_float2(-a.x, -a.y); }
template <class V>
__device__ __forceinline__ V vsqrt(V a);
template <> __device__ __forceinline__ float vsqrt<float>(float a) { return __fsqrt_rn(a); }
template <> __device__ __forceinline__ float2 vsqrt<float2>(float2 a) { return make_float2(__fsqrt_rn(a.x), __fsqrt_rn(a.y)); }

template <class V>
__device__ __forceinline__ void collide_srt_smag_v(V h[27], V Fx, V Fy, V Fz, float tau0, float smag_c2, V& drho_o,
                                                   V& jx_o, V& jy_o, V& jz_o)
{
    using P = typename ZPair<V>::T;
    P hp[9];
    V hs[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        hp[r] = zmk(h[r], h[18 + r]);
        hs[r] = h[9 + r];
    }
    const MomentsV<V> M = raw_moments_paired<V>(hp, hs);
    const V rho = sadd(vc<V>(1.0f), M.drho);
    const V inv = vrcp(rho);
    const V half = vc<V>(0.5f);
    const V ux = smul(sfma(half, Fx, M.jx), inv);
    const V uy = smul(sfma(half, Fy, M.jy), inv);
    const V uz = smul(sfma(half, Fz, M.jz), inv);
    const V nux = sneg(ux), nuy = sneg(uy), nuz = sneg(uz);
    const V rux = smul(rho, ux), ruy = smul(rho, uy);
    const V mt = vc<V>(-1.0f / 3.0f);
    // non-equilibrium second moments: S_ab - rho/3 delta - rho u_a u_b + (u_a F_b + u_b F_a)/2
    const V axx = sfma(ux, Fx, sfma(rux, nux, sfma(M.drho, mt, M.Sxx)));
    const V ayy = sfma(uy, Fy, sfma(ruy, nuy, sfma(M.drho, mt, M.Syy)));
    const V azz = sfma(uz, Fz, sfma(smul(rho, uz), nuz, sfma(M.drho, mt, M.Szz)));
    const V axy = sfma(half, sfma(ux, Fy, smul(uy, Fx)), sfma(rux, nuy, M.Sxy));
    const V axz = sfma(half, sfma(ux, Fz, smul(uz, Fx)), sfma(rux, nuz, M.Sxz));
    const V ayz = sfma(half, sfma(uy, Fz, smul(uz, Fy)), sfma(ruy, nuz, M.Syz));
    const V off = sfma(axy, axy, sfma(axz, axz, smul(ayz, ayz)));
    const V P2 = sfma(axx, axx, sfma(ayy, ayy, sfma(azz, azz, sadd(off, off))));
    const V arg = sfma(smul(vc<V>(18.0f * 1.41421356237f * smag_c2), vsqrt(P2)), inv, vc<V>(tau0 * tau0));
    const V tau = smul(half, sadd(vc<V>(tau0), vsqrt(arg)));
    const V om = vrcp(tau);
    const V src = sfma(om, vc<V>(-0.5f), vc<V>(1.0f));
    const V uu = sfma(ux, ux, sfma(uy, uy, smul(uz, uz)));
    const V uF = sfma(ux, Fx, sfma(uy, Fy, smul(uz, Fz)));
    // h* = (1 - om) h + om feq + S, evaluated for each pair q, qbar = 26 - q
    // together: c.u and c.F change sign with c, so om feq + S splits into a part
    // even in c, w (om (drho + rho (4.5 (c.u)^2 - 1.5 u^2)) + src (9 (c.u)(c.F) - 3 u.F)),
    // and an odd part, w 3 (om rho c.u + src c.F); c.u and c.F are formed for
    // the member of the pair whose first nonzero component (z, then y, then x)
    // is +1, so the sums start without a sign change
    const V a = ssub(vc<V>(1.0f), om);
    const V om_rho = smul(om, rho);
    const V k1 = smul(vc<V>(4.5f), om_rho);
    const V s9 = smul(vc<V>(9.0f), src);
    const V k0 = sfma(smul(vc<V>(-1.5f), om_rho), uu, sfma(om, M.drho, smul(smul(vc<V>(-3.0f), src), uF)));
    auto dot = [](int cx, int cy, int cz, V x, V y, V z) {
        V r = cz != 0 ? z : (cy != 0 ? y : x);  // the first nonzero component, +1
        if (cz != 0 && cy != 0) r = cy > 0 ? sadd(r, y) : ssub(r, y);
        if ((cz != 0 || cy != 0) && cx != 0) r = cx > 0 ? sadd(r, x) : ssub(r, x);
        return r;
    };
#pragma unroll
    for (int p = 0; p < 13; ++p) {
        const int q = 26 - p;  // c_q = -c_p, first nonzero component +1
        const V cu = dot(qcx(q), qcy(q), qcz(q), ux, uy, uz);
        const V cF = dot(qcx(q), qcy(q), qcz(q), Fx, Fy, Fz);
        const V pe = smul(vc<V>(wq(q)), sfma(cu, sfma(k1, cu, smul(s9, cF)), k0));
        const V po = smul(vc<V>(3.0f * wq(q)), sfma(om_rho, cu, smul(src, cF)));
        h[q] = sfma(a, h[q], sadd(pe, po));
        h[p] = sfma(a, h[p], ssub(pe, po));
    }
    h[13] = sfma(a, h[13], smul(vc<V>(wq(13)), k0));
    drho_o = M.drho;
    jx_o = sadd(M.jx, Fx);
    jy_o = sadd(M.jy, Fy);
    jz_o = sadd(M.jz, Fz);
}

// One cell (the form every kernel but the paired bulk kernel uses).
__device__ __forceinline__ void collide_srt_smag(float h[27], float Fx, float Fy, float Fz, float tau0, float smag_c2,
                                                 float& drho_o, float& jx_o, float& jy_o, float& jz_o)
{
    collide_srt_smag_v<float>(h, Fx, Fy, Fz, tau0, smag_c2, drho_o, jx_o, jy_o, jz_o);
}

// ------------------------------------------------------------------ streaming

__device__ __forceinline__ long long cell_of(const DevDomain* D, int x, int y, int z)
{
    return ((long long)z * D->ny + y) * D->nx + x;
}

// Wall rules for a cell next to a no-slip or free-slip face, applied after the
// clamped loads of k_step (out of line: wall cells are few).  For every
// direction q whose source x - c_q lies outside the lattice:
//   - no-slip axis: halfway bounce-back, the cell's own post-collision
//     population of the opposite direction (checked first);
//   - free-slip axis: specular reflection, the mirrored direction (that
//     component negated) read at the source moved back onto the cell's own
//     index along that axis; the other axes wrap, or meet the x inlet (the
//     mirrored direction's inlet equilibrium) or outlet (clamp).
template <typename T>
__device__ __noinline__ void boundary_patch(const DevDomain* D, const T* src, int x, int y, int z, long long step,
                                            float* h)
{
    const int n[3] = {D->nx, D->ny, D->nz};
    const int p[3] = {x, y, z};
    const unsigned cell = (unsigned)(((long long)z * D->ny + y) * D->nx + x);
    const unsigned N = (unsigned)D->N;
    for (int q = 0; q < 27; ++q) {
        const int c[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
        int s[3], cm[3];
        bool wall = false, reflected = false;
        for (int a = 0; a < 3; ++a) {
            s[a] = p[a] - c[a];
            cm[a] = c[a];
            if (D->bc[a] == BC_NOSLIP && (s[a] < 0 || s[a] >= n[a])) wall = true;
        }
        if (wall) {
            h[q] = Io<T>::ld(src + (unsigned)(26 - q) * N + cell);
            continue;
        }
        for (int a = 0; a < 3; ++a)
            if (D->bc[a] == BC_FREESLIP && (s[a] < 0 || s[a] >= n[a])) {
                cm[a] = -c[a];
                s[a] = p[a];
                reflected = true;
            }
        if (!reflected) continue;
        const int qm = (cm[2] + 1) * 9 + (cm[1] + 1) * 3 + (cm[0] + 1);
        for (int a = 0; a < 3; ++a)
            if (D->bc[a] == BC_PERIODIC) s[a] = s[a] < 0 ? s[a] + n[a] : (s[a] >= n[a] ? s[a] - n[a] : s[a]);
        if (D->bc[0] == BC_INOUT) {
            if (s[0] < 0) {  // the mirrored direction still has c_x = +1: a ghost population
                const float* gb = D->inflow_ghost[step & 1];
                h[q] = gb[((cm[2] + 1) * 3 + (cm[1] + 1)) * (D->ny * D->nz) + s[2] * D->ny + s[1]];
                continue;
            }
            if (s[0] >= n[0]) s[0] = n[0] - 1;
        }
        h[q] = Io<T>::ld(src + (unsigned)qm * N + (unsigned)(((long long)s[2] * D->ny + s[1]) * D->nx + s[0]));
    }
}

// ------------------------------------------------------------------ actuator line

// Segment of an ascending table containing x (x strictly inside the range):
// direct index for equally spaced tables, bisection otherwise.
__device__ __forceinline__ int table_segment(const DevTurbine* B, float x)
{
    const float* xs = B->alpha;
    const int n = B->n_polar;
    int lo;
    if (B->polar_uniform) {
        lo = (int)floorf((x - B->polar_a0) * B->polar_inv_da);
        lo = lo < 0 ? 0 : (lo > n - 2 ? n - 2 : lo);
        while (lo > 0 && xs[lo] > x) --lo;
        while (lo < n - 2 && xs[lo + 1] < x) ++lo;
    } else {
        lo = 0;
        int hi = n - 1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (xs[mid] <= x) lo = mid; else hi = mid;
        }
    }
    return lo;
}

// C_L and C_D at angle of attack x: linear interpolation, clamped at the ends.
__device__ __forceinline__ void polar_lookup(const DevTurbine* B, float x, float& CL, float& CD)
{
    const float* xs = B->alpha;
    const int n = B->n_polar;
    if (x <= xs[0]) { CL = B->cl[0]; CD = B->cd[0]; return; }
    if (x >= xs[n - 1]) { CL = B->cl[n - 1]; CD = B->cd[n - 1]; return; }
    const int lo = table_segment(B, x);
    const float t = (x - xs[lo]) / (xs[lo + 1] - xs[lo]);
    CL = B->cl[lo] + t * (B->cl[lo + 1] - B->cl[lo]);
    CD = B->cd[lo] + t * (B->cd[lo + 1] - B->cd[lo]);
}

// Sum of the ALM force boxes containing cell (x, y, z): the force of the last
// collision (read through L2).
__device__ __forceinline__ void alm_box_force(const DevDomain* D, int x, int y, int z, float F[3])
{
    for (int t = 0; t < D->n_turb; ++t) {
        const DevTurbine* B = D->turb + t;
        if (x < B->lo[0] || x > B->hi[0] || y < B->lo[1] || y > B->hi[1] || z < B->lo[2] || z > B->hi[2]) continue;
        const long long bi = ((long long)(z - B->lo[2]) * B->bny + (y - B->lo[1])) * B->bnx + (x - B->lo[0]);
        F[0] += __ldcg(B->fbox + bi);
        F[1] += __ldcg(B->fbox + B->bcells + bi);
        F[2] += __ldcg(B->fbox + 2 * B->bcells + bi);
    }
}

// Geometry of blade element g at step n (Algorithm 2 for a hub + straight
// blades): blade angle theta = theta0 + omega n + 2 pi b / B accumulated in
// FP64 from the integer step and reduced mod 2 pi, then FP32.
struct ElementGeo {
    const DevTurbine* B;
    int k;
    float r, len;
    float p[3], v[3], er[3], et[3];
};

__device__ __forceinline__ void element_geometry(const DevDomain* D, int g, long long step, ElementGeo& G)
{
    int t = 0;
    while (t + 1 < D->n_turb && D->turb[t + 1].el_offset <= g) ++t;
    const DevTurbine* B = D->turb + t;
    const int le = g - B->el_offset;
    const int b = le / B->n_elements;
    G.B = B;
    G.k = le - b * B->n_elements;
    double th = B->theta0 + B->omega * (double)step + 6.283185307179586 * (double)b / (double)B->n_blades;
    th = fmod(th, 6.283185307179586);
    float sn, cs;
    sincosf((float)th, &sn, &cs);
    const float* ea = B->e_axis;
#pragma unroll
    for (int a = 0; a < 3; ++a) G.er[a] = cs * B->e1[a] + sn * B->e2[a];
    G.et[0] = ea[1] * G.er[2] - ea[2] * G.er[1];
    G.et[1] = ea[2] * G.er[0] - ea[0] * G.er[2];
    G.et[2] = ea[0] * G.er[1] - ea[1] * G.er[0];
    G.len = B->radius / (float)B->n_elements;
    G.r = ((float)G.k + 0.5f) * G.len;
    const float om = (float)B->omega;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        G.p[a] = B->hub[a] + G.r * G.er[a];
        G.v[a] = om * G.r * G.et[a];
    }
}

// Three-point discrete delta of Roma, Peskin and Berger (1999), the spreading
// kernel of Sec. 2.2: (1 + sqrt(1 - 3 r^2)) / 3 for |r| <= 1/2,
// (5 - 3|r| - sqrt(1 - 3 (1 - |r|)^2)) / 6 for 1/2 < |r| <= 3/2, else 0.
__device__ __forceinline__ float roma_phi(float r)
{
    const float a = fabsf(r);
    if (a <= 0.5f) return (1.0f + sqrtf(1.0f - 3.0f * a * a)) * (1.0f / 3.0f);
    if (a <= 1.5f) {
        const float b = 1.0f - a;
        return (5.0f - 3.0f * a - sqrtf(fmaxf(1.0f - 3.0f * b * b, 0.0f))) * (1.0f / 6.0f);
    }
    return 0.0f;
}

// Glauert's tip-loss factor in Prandtl's form (Sec. 2.2): for B blades of
// radius R, an element at radius r with inflow angle phi,
// (2/pi) arccos(exp(-B (R - r) / (2 r |sin phi|))); 1 where sin phi = 0.
__device__ __forceinline__ float tip_loss_factor(int n_blades, float R, float r, float phi)
{
    const float s = fabsf(sinf(phi));
    if (s == 0.0f) return 1.0f;
    const float f = (float)n_blades * (R - r) / (2.0f * r * s);
    return 0.63661977f * acosf(expf(-f));  // 2/pi
}

// Normaliser of an element's spreading kernel at position p: the product over
// the axes of the sums of the kernel's weights over the lattice points within
// the cut (exp(-(i - p)^2 / eps^2) for the Gaussian; 1 up to rounding for Roma).
__device__ __forceinline__ float spread_norm(const DevTurbine* B, const float p[3])
{
    float S = 1.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int lo = (int)ceilf(p[a] - B->cut), hi = (int)floorf(p[a] + B->cut);
        float sa = 0.0f;
        if (B->roma) {
            for (int j = lo; j <= hi; ++j) sa += roma_phi((float)j - p[a]);
        } else {
            for (int j = lo; j <= hi; ++j) {
                const float d = (float)j - p[a];
                sa += expf(-d * d * B->inv_eps2);
            }
        }
        S *= sa;
    }
    return S;
}

// Actuator line of step `step` for the blade elements [e0, e0 + kAlmBlock) of
// one lattice, by the whole CTA.  Reads the populations of the current array f
// (post-collision of step-1) and the box force of step-1; writes the element
// positions with their spreading normalisation, blade forces and FP64 load
// parts of those elements into the buffers of parity step & 1.
//  phase 0, one thread per element: blade kinematics (Algorithm 2) and the
//    kernel normaliser, which depend on the step alone;
//  then, in a dependent launch, the wait for the launch before it (the rotor
//    tiles, which write the cells sampled below and the box force);
//  phase 1, one thread per (element, corner): pull the 27 populations of the
//    corner cell, rho and u = (sum c f + F/2)/rho at the corner;
//  phase 2, one thread per element: trilinear blend, relative velocity,
//    angle of attack, polars, blade force (with the tip-loss factor if set),
//    FP64 load parts.
// Each element's values depend on that element alone, so blocks of elements
// may run in separate CTAs.
template <typename T>
__device__ __noinline__ void alm_block(const DevDomain* D, const T* f, long long step, int swapped, int e0)
{
    __shared__ ElementGeo s_geo[kAlmBlock];
    __shared__ float s_norm[kAlmBlock];
    __shared__ float4 s_corner[8 * kAlmBlock];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    const int par = (int)(step & 1);
    const long long N = D->N;
    const int n[3] = {D->nx, D->ny, D->nz};
    const int ne = min(kAlmBlock, D->n_el - e0);
    for (int i = tid; i < ne; i += nthr) {
        element_geometry(D, e0 + i, step, s_geo[i]);
        s_norm[i] = spread_norm(s_geo[i].B, s_geo[i].p);
    }
    __syncthreads();
    // a no-op outside a dependent launch
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int pc = tid; pc < 8 * ne; pc += nthr) {
        const int i = pc >> 3, cn = pc & 7;
        int c[3];
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int i0 = (int)floorf(s_geo[i].p[a]);
            if (i0 < 1 || i0 + 1 > n[a] - 2) inside = false;
            c[a] = i0 + ((cn >> a) & 1);
        }
        float4 out = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
        if (inside) {
            // pulled populations of the corner cell: the pull sources, or (in-place
            // array after an even step) the cell's own opposite slots
            float h[27];
            if (swapped) {
                const long long cc = cell_of(D, c[0], c[1], c[2]);
#pragma unroll
                for (int q = 0; q < 27; ++q) h[q] = Io<T>::ldcg(f + (size_t)(26 - q) * N + cc);
            } else {
#pragma unroll
                for (int q = 0; q < 27; ++q)
                    h[q] = Io<T>::ldcg(f + (size_t)q * N + cell_of(D, c[0] - qcx(q), c[1] - qcy(q), c[2] - qcz(q)));
            }
            float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                drho += h[q];
                jx += (float)qcx(q) * h[q];
                jy += (float)qcy(q) * h[q];
                jz += (float)qcz(q) * h[q];
            }
            float F[3] = {D->body[0], D->body[1], D->body[2]};
            alm_box_force(D, c[0], c[1], c[2], F);
            const float rho = 1.0f + drho;
            out = make_float4(rho, (jx + 0.5f * F[0]) / rho, (jy + 0.5f * F[1]) / rho, (jz + 0.5f * F[2]) / rho);
        } else if (cn == 0) {
            atomicOr(D->err, ERR_ELEMENT_OUTSIDE);
        }
        s_corner[pc] = out;
    }
    __syncthreads();
    for (int i = tid; i < ne; i += nthr) {
        const int g = e0 + i;
        const ElementGeo G = s_geo[i];
        const DevTurbine* B = G.B;
        float fr[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) fr[a] = G.p[a] - floorf(G.p[a]);
        float rho_p = 0.f, u_p[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int cn = 0; cn < 8; ++cn) {
            const float w = ((cn & 1) ? fr[0] : 1.0f - fr[0]) * (((cn >> 1) & 1) ? fr[1] : 1.0f - fr[1]) *
                            (((cn >> 2) & 1) ? fr[2] : 1.0f - fr[2]);
            const float4 q = s_corner[8 * i + cn];
            rho_p += w * q.x;
            u_p[0] += w * q.y;
            u_p[1] += w * q.z;
            u_p[2] += w * q.w;
        }
        // relative velocity without its radial part, angle of attack, polars
        const float* ea = B->e_axis;
        float ur[3] = {u_p[0] - G.v[0], u_p[1] - G.v[1], u_p[2] - G.v[2]};
        const float urad = ur[0] * G.er[0] + ur[1] * G.er[1] + ur[2] * G.er[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) ur[a] -= urad * G.er[a];
        const float uax = ur[0] * ea[0] + ur[1] * ea[1] + ur[2] * ea[2];
        const float utan = ur[0] * G.et[0] + ur[1] * G.et[1] + ur[2] * G.et[2];
        const float phi = atan2f(uax, -utan);
        const float twist = B->twist ? B->twist[G.k] : 0.0f;
        const float alpha = phi - twist - B->pitch;
        float CL, CD;
        polar_lookup(B, alpha, CL, CD);
        const float chord = B->chord_root + (B->chord_tip - B->chord_root) * G.r / B->radius;
        const float mag2 = ur[0] * ur[0] + ur[1] * ur[1] + ur[2] * ur[2];
        float Fb[3] = {0.0f, 0.0f, 0.0f};
        if (mag2 > 0.0f) {
            const float mag = sqrtf(mag2);
            const float eD[3] = {ur[0] / mag, ur[1] / mag, ur[2] / mag};
            const float eL[3] = {eD[1] * G.er[2] - eD[2] * G.er[1], eD[2] * G.er[0] - eD[0] * G.er[2],
                                 eD[0] * G.er[1] - eD[1] * G.er[0]};
            float sc = 0.5f * rho_p * mag2 * chord * G.len;
            if (B->tip_loss) sc *= tip_loss_factor(B->n_blades, B->radius, G.r, phi);
#pragma unroll
            for (int a = 0; a < 3; ++a) Fb[a] = sc * (CL * eL[a] + CD * eD[a]);
        }
        const float S = s_norm[i];
        D->el_pos[par][g] = make_float4(G.p[0], G.p[1], G.p[2], 1.0f / S);
        D->el_force[par][g] = make_float4(Fb[0], Fb[1], Fb[2], alpha);
        D->el_load[2 * g] = (double)Fb[0] * ea[0] + (double)Fb[1] * ea[1] + (double)Fb[2] * ea[2];
        D->el_load[2 * g + 1] =
            (double)G.r * ((double)Fb[0] * G.et[0] + (double)Fb[1] * G.et[1] + (double)Fb[2] * G.et[2]);
    }
    __syncthreads();
}

// Per-rotor FP64 thrust and torque of step `step` from the elements' load
// parts, by warp 0 of the CTA in a fixed order (lane-strided partial sums, then
// a butterfly), also written to the host loads sink when one is set.
__device__ __forceinline__ void alm_loads(const DevDomain* D, long long step)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int par = (int)(step & 1);
    if (tid < 32) {
        for (int t = 0; t < D->n_turb; ++t) {
            const DevTurbine* B = D->turb + t;
            const int ne = B->n_blades * B->n_elements;
            double th = 0.0, tq = 0.0;
            for (int e = tid; e < ne; e += 32) {
                th += __ldcg(D->el_load + 2 * (B->el_offset + e));
                tq += __ldcg(D->el_load + 2 * (B->el_offset + e) + 1);
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                th += __shfl_xor_sync(0xFFFFFFFFu, th, o);
                tq += __shfl_xor_sync(0xFFFFFFFFu, tq, o);
            }
            if (tid == 0) {
                D->loads[par][2 * t] = th;
                D->loads[par][2 * t + 1] = tq;
                if (D->loads_sink) {  // zero-copy to the caller's host ring
                    double* o = D->loads_sink + 2 * ((step % D->sink_len) * D->n_turb + t);
                    o[0] = th;
                    o[1] = tq;
                }
            }
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ the time step

// A work-list entry, read with an L2 evict-last policy: the list is read once per
// step among the PDF streams, and without the hint it would be evicted and
// cost every CTA a DRAM round trip before its first PDF load.
__device__ __forceinline__ unsigned long long ld_tile(const unsigned long long* p)
{
    unsigned long long v, pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
    return v;
}

// Pulled pre-collision populations of cell (x, y, z): clamped/wrapped loads,
// then the inlet and wall rules (WALLS false: the lattices have no no-slip or
// free-slip face, and the wall code is left out).
template <typename T, bool WALLS = true>
__device__ __forceinline__ void load_cell(const DevDomain* D, const T* __restrict__ src, int x, int y, int z,
                                          long long step, float h[27])
{
    const int nx = D->nx, ny = D->ny, nz = D->nz;
    // source coordinates for c = +1 (m) and c = -1 (p): wrapped on periodic
    // axes, clamped otherwise (the outlet rule; other faces are patched below)
    const int bx = D->bc[0], by = D->bc[1], bz = D->bc[2];
    int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
    if (bx == BC_PERIODIC) { if (xm < 0) xm += nx; if (xp >= nx) xp -= nx; }
    else { xm = max(xm, 0); xp = min(xp, nx - 1); }
    if (by == BC_PERIODIC) { if (ym < 0) ym += ny; if (yp >= ny) yp -= ny; }
    else { ym = max(ym, 0); yp = min(yp, ny - 1); }
    if (bz == BC_PERIODIC) { if (zm < 0) zm += nz; if (zp >= nz) zp -= nz; }
    else { zm = max(zm, 0); zp = min(zp, nz - 1); }
    const bool walls = WALLS && (((bx == BC_NOSLIP || bx == BC_FREESLIP) && (x == 0 || x == nx - 1)) ||
                                 ((by == BC_NOSLIP || by == BC_FREESLIP) && (y == 0 || y == ny - 1)) ||
                                 ((bz == BC_NOSLIP || bz == BC_FREESLIP) && (z == 0 || z == nz - 1)));
    // 32-bit offsets: 27 N < 2^31 is checked on the host
    const unsigned uN = (unsigned)D->N;
    const unsigned xs[3] = {(unsigned)xp, (unsigned)x, (unsigned)xm};  // source x for cx = -1, 0, +1
    const unsigned ys[3] = {(unsigned)yp, (unsigned)y, (unsigned)ym};
    const unsigned zs[3] = {(unsigned)zp, (unsigned)z, (unsigned)zm};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const unsigned row = (zs[k] * (unsigned)ny + ys[j]) * (unsigned)nx;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int q = k * 9 + j * 3 + i;
                h[q] = Io<T>::ld(src + ((unsigned)q * uN + row + xs[i]));
            }
        }
    // x inlet: the nine directions with c_x = +1 come from the ghost column
    // (y - c_y, z - c_z): equilibrium at rho = 1 and that column's inlet velocity,
    // precomputed per column in the ghost buffer
    if (bx == BC_INOUT && x == 0) {
        const float* gb = D->inflow_ghost[step & 1];
        const int plane = ny * nz;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int q = k * 9 + j * 3 + 2;
                const bool wall = WALLS && ((by == BC_NOSLIP && ((j == 2 && y == 0) || (j == 0 && y == ny - 1))) ||
                                            (bz == BC_NOSLIP && ((k == 2 && z == 0) || (k == 0 && z == nz - 1))));
                if (!wall) h[q] = gb[(k * 3 + j) * plane + (int)zs[k] * ny + (int)ys[j]];
            }
    }
    if (WALLS && walls) {
        float hl[27];
#pragma unroll
        for (int q = 0; q < 27; ++q) hl[q] = h[q];
        boundary_patch<T>(D, src, x, y, z, step, hl);
#pragma unroll
        for (int q = 0; q < 27; ++q) h[q] = hl[q];
    }
}

// Regularised force of rotor t at cell (x, y, z): the sum over its elements in
// element order (from the culled list when it fits) of -w F_e, with w the
// Gaussian exp(-|d|^2 / eps^2) (ROMA false) or the product of Roma's delta
// (ROMA true) times the element's normaliser.  The kernel is a template
// argument so that the pair loop carries no per-pair branch on it.
template <bool ROMA>
__device__ __forceinline__ void gather_rotor(const DevTurbine* B, int t, int x, int y, int z, int n_cull,
                                             const float4* s_pos, const float4* s_frc, const int* s_tag,
                                             const float4* P, const float4* Fe, float& ax, float& ay, float& az)
{
    const float cut = B->cut, ie2 = B->inv_eps2;
    auto add = [&](float4 pe, float4 fe_or_none, bool from_list, int e) {
        const float dx = (float)x - pe.x, dy = (float)y - pe.y, dz = (float)z - pe.z;
        if (fabsf(dx) <= cut && fabsf(dy) <= cut && fabsf(dz) <= cut) {
            const float w = (ROMA ? roma_phi(dx) * roma_phi(dy) * roma_phi(dz)
                                  : expf(-(dx * dx + dy * dy + dz * dz) * ie2)) * pe.w;
            const float4 fe = from_list ? fe_or_none : __ldg(Fe + B->el_offset + e);
            ax -= w * fe.x;
            ay -= w * fe.y;
            az -= w * fe.z;
        }
    };
    if (n_cull >= 0) {
        for (int i = 0; i < n_cull; ++i)
            if (s_tag[i] == t) add(s_pos[i], s_frc[i], true, 0);
    } else {
        const int ne = B->n_blades * B->n_elements;
        for (int e = 0; e < ne; ++e) add(__ldg(P + B->el_offset + e), make_float4(0.f, 0.f, 0.f, 0.f), false, e);
    }
}

// Regularised blade force at cell (x, y, z) of a rotor tile, summed over the
// rotors whose box holds the cell; each rotor's part is stored in its force box.
__device__ __forceinline__ void rotor_force(const DevDomain* D, long long step, int x, int y, int z, int n_cull,
                                            const float4* s_pos, const float4* s_frc, const int* s_tag, float F[3])
{
    const float4* P = D->el_pos[step & 1];
    const float4* Fe = D->el_force[step & 1];
    for (int t = 0; t < D->n_turb; ++t) {
        const DevTurbine* B = D->turb + t;
        if (x < B->lo[0] || x > B->hi[0] || y < B->lo[1] || y > B->hi[1] || z < B->lo[2] || z > B->hi[2]) continue;
        float ax = 0.0f, ay = 0.0f, az = 0.0f;
        if (B->roma)
            gather_rotor<true>(B, t, x, y, z, n_cull, s_pos, s_frc, s_tag, P, Fe, ax, ay, az);
        else
            gather_rotor<false>(B, t, x, y, z, n_cull, s_pos, s_frc, s_tag, P, Fe, ax, ay, az);
        const long long bi = ((long long)(z - B->lo[2]) * B->bny + (y - B->lo[1])) * B->bnx + (x - B->lo[0]);
        B->fbox[bi] = ax;
        B->fbox[B->bcells + bi] = ay;
        B->fbox[2 * B->bcells + bi] = az;
        F[0] += ax;
        F[1] += ay;
        F[2] += az;
    }
}

// Cull the blade elements whose support reaches the tile (planes [z0, z1)) into
// shared memory, in element order; returns their number, or -1 when more than
// KCULL reach it (every cell then scans all elements).  CTA-wide.
template <int KCULL>
__device__ __forceinline__ int cull_rotor_elements(const DevDomain* D, unsigned long long tile, long long step, int z0,
                                                   int z1, float4* s_pos, float4* s_frc, int* s_tag, int* s_cnt)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    const float tx0 = (float)(tile & 0xFFFF), ty0 = (float)((tile >> 16) & 0xFFFF);
    const float tx1 = tx0 + (float)(blockDim.x - 1), ty1 = ty0 + (float)(blockDim.y - 1);
    const float tz0 = (float)z0, tz1 = (float)(z1 - 1);
    const float4* P = D->el_pos[step & 1];
    const float4* Fe = D->el_force[step & 1];
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
    int total = 0;
    for (int base = 0; base < D->n_el; base += nthreads) {
        const int e = base + tid;
        bool keep = false;
        float4 pe = make_float4(0.f, 0.f, 0.f, 0.f);
        int t = 0;
        if (e < D->n_el) {
            pe = __ldg(P + e);
            while (t + 1 < D->n_turb && D->turb[t + 1].el_offset <= e) ++t;
            const float cut = D->turb[t].cut;
            keep = pe.x + cut >= tx0 && pe.x - cut <= tx1 && pe.y + cut >= ty0 && pe.y - cut <= ty1 &&
                   pe.z + cut >= tz0 && pe.z - cut <= tz1;
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
        if (lane == 0) s_cnt[warp] = __popc(m);
        __syncthreads();
        int off = total, chunk = 0;
        for (int w = 0; w < nwarps; ++w) {
            if (w < warp) off += s_cnt[w];
            chunk += s_cnt[w];
        }
        const int pos = off + __popc(m & ((1u << lane) - 1u));
        if (keep && pos < KCULL) {
            s_pos[pos] = pe;
            s_frc[pos] = __ldg(Fe + e);
            s_tag[pos] = t;
        }
        total += chunk;
        __syncthreads();
    }
    return total <= KCULL ? total : -1;
}

// The update of one rotor tile: cull the blade elements whose support reaches
// the tile into shared memory (in element order; when more than KCULL reach it
// every cell scans all elements), then each cell as in the bulk path plus the
// regularised blade force (Gaussian or Roma).  CTA-wide; only the rotor launch
// of k_step contains it.  Writes the thread's diagnostic partial sums (zero
// unless diag) to sums[4].
template <int COLL, typename T, bool MARCH, int KCULL>
__device__ __forceinline__ void rotor_tile_update(const DevDomain* D, unsigned long long tile, long long step, int parity,
                                               int planes, bool diag, float4* s_pos, float4* s_frc, int* s_tag,
                                               int* s_cnt, double* sums)
{
    const int z0 = (int)((tile >> 32) & 0xFFFF);
    const int y = (int)((tile >> 16) & 0xFFFF) + threadIdx.y;
    const int x = (int)(tile & 0xFFFF) + threadIdx.x;
    const int nx = D->nx, ny = D->ny, nz = D->nz;
    const int z1 = MARCH ? min(z0 + planes, nz) : z0 + 1;  // planes [z0, z1)
    const unsigned uN = (unsigned)D->N;
    const T* __restrict__ src = (const T*)D->f[parity];
    T* __restrict__ dst = (T*)D->f[parity ^ 1];

    const int n_cull = cull_rotor_elements<KCULL>(D, tile, step, z0, z1, s_pos, s_frc, s_tag, s_cnt);

    // diagnostic partial sums of the thread's planes (diagnostic steps only),
    // in FP64 when it marches over several planes
    using Acc = typename std::conditional<MARCH, double, float>::type;
    Acc o_m = 0, o_jx = 0, o_jy = 0, o_jz = 0;
    if (x < nx && y < ny) {
        float hn[27];
        load_cell<T>(D, src, x, y, z0, step, hn);
#pragma unroll 1
        for (int z = z0; z < z1; ++z) {
            float h[27];
#pragma unroll
            for (int q = 0; q < 27; ++q) h[q] = hn[q];
            if (MARCH && z + 1 < z1) load_cell<T>(D, src, x, y, z + 1, step, hn);
            if (D->bc[0] == BC_INOUT && x == 0) write_inlet_ghost(D, step + 1, y, z);
            float F[3] = {D->body[0], D->body[1], D->body[2]};
            rotor_force(D, step, x, y, z, n_cull, s_pos, s_frc, s_tag, F);
            float m, jx, jy, jz;
            if (COLL == COLL_CUMULANT)
                collide_cumulant(h, F[0], F[1], F[2], D->omega, m, jx, jy, jz);
            else
                collide_srt_smag(h, F[0], F[1], F[2], D->tau0, D->smag_c2, m, jx, jy, jz);
            if (diag) {
                o_m += m;
                o_jx += jx;
                o_jy += jy;
                o_jz += jz;
            }
            const unsigned cell = ((unsigned)z * (unsigned)ny + (unsigned)y) * (unsigned)nx + (unsigned)x;
#pragma unroll
            for (int q = 0; q < 27; ++q) Io<T>::st(dst + ((unsigned)q * uN + cell), h[q]);
        }
    }
    sums[0] = (double)o_m;
    sums[1] = (double)o_jx;
    sums[2] = (double)o_jy;
    sums[3] = (double)o_jz;
}

// One time step over the work list, as two launches of this kernel: ROTOR over
// the rotor tiles, then the rest (almost all of the lattice), whose code then
// carries none of the rotor path.  A CTA covers tile_x x tile_y cells of tile_z
// consecutive planes; with MARCH a thread walks its column of planes and issues
// the loads of the next plane before the collision of the current one.
// The CTA's diagnostic partial sums (mass and momentum of its cells) into the
// lattice's FP64 accumulators; the last CTA of the step, counted over all its
// launches, publishes every lattice's sums with the step and flags non-finite
// ones.  CTA-wide, on diagnostic steps only.
__device__ __forceinline__ void diag_close(const StepArgs& A, const DevDomain* D, long long step, double m, double jx,
                                           double jy, double jz, double (*s_red)[4])
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    double v[4] = {m, jx, jy, jz};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v[k] += __shfl_xor_sync(0xFFFFFFFFu, v[k], o);
    if ((tid & 31) == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) s_red[tid >> 5][k] = v[k];
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < 4; ++k) {
            double sum = 0.0;
            for (int w = 0; w < (nthreads >> 5); ++w) sum += s_red[w][k];
            atomicAdd(D->diag_acc + k, sum);
        }
        __threadfence();
        const unsigned prev = atomicAdd(A.diag_done, 1u);
        if (prev == A.n_total - 1u) {
            __threadfence();
            for (int i = 0; i < A.n_inst; ++i) {
                const DevDomain* Di = A.dom + i;
                bool finite = true;
                for (int k = 0; k < 4; ++k) {
                    const double sum = __ldcg(Di->diag_acc + k);
                    Di->diag_res[k] = sum;
                    Di->diag_acc[k] = 0.0;
                    if (!isfinite(sum)) finite = false;
                }
                Di->diag_res[4] = (double)step;
                if (!finite) atomicOr(Di->err, ERR_NONFINITE);
            }
            *A.diag_done = 0u;
        }
    }
}

// The rotor CTAs allow the dependent launch (the actuator line, whose CTAs do
// the same for the bulk) to start as soon as they are all running, so the
// bulk overlaps the rotor tiles and the actuator line of the next step.  The
// launches write disjoint cells.  Each launch's last CTA waits for the launch
// before it before it exits, so the bulk launch ends only after all of them.
// Register budgets (blocks of up to 256 threads): 64 per thread for the
// single-plane cumulant bulk, whose collision fits them without spills, so 8
// CTAs of 128 threads (32 warps) are resident per SM; 85 for the rotor tiles
// and the Smagorinsky collision; 128 for marching, which holds two planes.
template <int COLL, typename T, bool MARCH, bool ROTOR, bool WALLS = true>
__global__ void __launch_bounds__(256, MARCH ? 2 : ((ROTOR || COLL != COLL_CUMULANT) ? 3 : 4)) k_step(const StepArgs A)
{
    if (ROTOR || A.trigger) asm volatile("griddepcontrol.launch_dependents;");
    constexpr int kCull = 128;  // blade elements kept per rotor tile
    __shared__ double s_red[8][4];
    __shared__ float4 s_pos[ROTOR ? kCull : 1], s_frc[ROTOR ? kCull : 1];
    __shared__ int s_tag[ROTOR ? kCull : 1];
    __shared__ int s_cnt[8];
    const unsigned long long tile = ld_tile(A.tiles + blockIdx.x);
    const int inst = tile_lattice(tile);
    const int z0 = (int)((tile >> 32) & 0xFFFF);
    const int y = (int)((tile >> 16) & 0xFFFF) + threadIdx.y;
    const int x = (int)(tile & 0xFFFF) + threadIdx.x;
    const DevDomain* D = A.dom + inst;
    const long long step = __ldcg(A.step_slot + A.parity);
    if (A.write_step && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        A.step_slot[A.parity ^ 1] = step + 1;
        A.diag_flag[A.parity ^ 1] = A.diag_every > 0 && (step + 1) % A.diag_every == 0;
    }
    const bool diag = __ldcg(A.diag_flag + A.parity) != 0;  // uniform over the grid
    // diagnostic partial sums of the thread's planes (diagnostic steps only),
    // in FP64 when it marches over several planes
    using Acc = typename std::conditional<MARCH, double, float>::type;
    Acc o_m = 0, o_jx = 0, o_jy = 0, o_jz = 0;

    if constexpr (ROTOR) {
        double sums[4];
        rotor_tile_update<COLL, T, MARCH, kCull>(D, tile, step, A.parity, tile_planes(tile), diag, s_pos, s_frc,
                                                 s_tag, s_cnt, sums);
        o_m = sums[0];
        o_jx = sums[1];
        o_jy = sums[2];
        o_jz = sums[3];
    } else {
        const int nx = D->nx, ny = D->ny, nz = D->nz;
        if (x < nx && y < ny) {
            const int z1 = MARCH ? min(z0 + A.tile_z, nz) : z0 + 1;  // planes [z0, z1)
            const unsigned uN = (unsigned)D->N;
            const T* __restrict__ src = (const T*)D->f[A.parity];
            T* __restrict__ dst = (T*)D->f[A.parity ^ 1];
            float hn[27];
            load_cell<T, WALLS>(D, src, x, y, z0, step, hn);
#pragma unroll 1
            for (int z = z0; z < z1; ++z) {
                float h[27];
#pragma unroll
                for (int q = 0; q < 27; ++q) h[q] = hn[q];
                if (MARCH && z + 1 < z1) load_cell<T, WALLS>(D, src, x, y, z + 1, step, hn);
                // the x = 0 lane of each row prepares the inlet ghost populations of its column for step n+1
                if (D->bc[0] == BC_INOUT && x == 0) write_inlet_ghost(D, step + 1, y, z);
                float m, jx, jy, jz;
                if (COLL == COLL_CUMULANT)
                    collide_cumulant(h, D->body[0], D->body[1], D->body[2], D->omega, m, jx, jy, jz);
                else
                    collide_srt_smag(h, D->body[0], D->body[1], D->body[2], D->tau0, D->smag_c2, m, jx, jy, jz);
                if (diag) {
                    o_m += m;
                    o_jx += jx;
                    o_jy += jy;
                    o_jz += jz;
                }
                const unsigned cell = ((unsigned)z * (unsigned)ny + (unsigned)y) * (unsigned)nx + (unsigned)x;
#pragma unroll
                for (int q = 0; q < 27; ++q) Io<T>::st(dst + ((unsigned)q * uN + cell), h[q]);
            }
        }
    }
    // diagnostic step (uniform over the grid): FP64 sums, closed by the last CTA
    if (diag) diag_close(A, D, step, o_m, o_jx, o_jy, o_jz, s_red);
    if constexpr (!ROTOR) {
        if (blockIdx.x == gridDim.x - 1) asm volatile("griddepcontrol.wait;" ::: "memory");
    }
}

// The bulk launch over the tiles with no cell on a no-slip or free-slip face
// (their other neighbours wrap on periodic axes or stay inside the lattice,
// and x may be an inlet/outlet), almost every cell of the workloads: the same
// update as k_step's bulk path, with the lattice's
// sizes, rates and array pointers read from the kernel parameters instead of
// its descriptor in global memory, and no wall code compiled in.  Inlet cells
// take their nine ghost populations from the inlet buffer.  DIAG: the host
// launches this form on diagnostic steps only (the sums' code costs the other
// steps even when it does not run); SINGLE: one lattice, whose parameters are
// then read at fixed offsets.
template <int COLL, typename T, bool DIAG, bool SINGLE>
__global__ void __launch_bounds__(256, 4) k_bulk(const StepArgs A, const BulkParams P)
{
    __shared__ double s_red[DIAG ? 8 : 1][4];
    const unsigned long long tile = ld_tile(A.tiles + blockIdx.x);
    const int inst = SINGLE ? 0 : tile_lattice(tile);
    const LatHot& L = P.lat[inst];
    const int z = (int)((tile >> 32) & 0xFFFF);
    const int y = (int)((tile >> 16) & 0xFFFF) + threadIdx.y;
    const int x = (int)(tile & 0xFFFF) + threadIdx.x;
    const long long step = __ldcg(A.step_slot + A.parity);
    if (A.write_step && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        A.step_slot[A.parity ^ 1] = step + 1;
        A.diag_flag[A.parity ^ 1] = A.diag_every > 0 && (step + 1) % A.diag_every == 0;
    }
    float o_m = 0.0f, o_jx = 0.0f, o_jy = 0.0f, o_jz = 0.0f;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    if (x < nx && y < ny) {
        const T* __restrict__ src = (const T*)L.f[A.parity];
        T* __restrict__ dst = (T*)L.f[A.parity ^ 1];
        const unsigned uN = L.N;
        int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
        if (L.inout) { xm = max(xm, 0); xp = min(xp, nx - 1); }  // outlet: zero-gradient clamp
        else { if (xm < 0) xm += nx; if (xp >= nx) xp -= nx; }
        if (ym < 0) ym += ny; if (yp >= ny) yp -= ny;
        if (zm < 0) zm += nz; if (zp >= nz) zp -= nz;
        const unsigned xs[3] = {(unsigned)xp, (unsigned)x, (unsigned)xm};
        const unsigned ys[3] = {(unsigned)yp, (unsigned)y, (unsigned)ym};
        const unsigned zs[3] = {(unsigned)zp, (unsigned)z, (unsigned)zm};
        float h[27];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const unsigned row = (zs[k] * (unsigned)ny + ys[j]) * (unsigned)nx;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int q = k * 9 + j * 3 + i;
                    h[q] = Io<T>::ld(src + ((unsigned)q * uN + row + xs[i]));
                }
            }
        if (L.inout && x == 0) {
            // the nine directions with c_x = +1 across the inlet face, from the ghost
            // columns (y - c_y, z - c_z); then this column's ghosts for step n+1
            const DevDomain* D = A.dom + inst;
            const float* gb = D->inflow_ghost[step & 1];
            const int plane = ny * nz;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int j = 0; j < 3; ++j) h[k * 9 + j * 3 + 2] = gb[(k * 3 + j) * plane + (int)zs[k] * ny + (int)ys[j]];
            write_inlet_ghost(D, step + 1, y, z);
        }
        float m, jx, jy, jz;
        if (COLL == COLL_CUMULANT)
            collide_cumulant(h, L.body[0], L.body[1], L.body[2], L.omega, m, jx, jy, jz);
        else
            collide_srt_smag(h, L.body[0], L.body[1], L.body[2], L.tau0, L.smag_c2, m, jx, jy, jz);
        if (DIAG) {
            o_m = m;
            o_jx = jx;
            o_jy = jy;
            o_jz = jz;
        }
        const unsigned cell = ((unsigned)z * (unsigned)ny + (unsigned)y) * (unsigned)nx + (unsigned)x;
#pragma unroll
        for (int q = 0; q < 27; ++q) Io<T>::st(dst + ((unsigned)q * uN + cell), h[q]);
    }
    if (DIAG) diag_close(A, A.dom + inst, step, o_m, o_jx, o_jy, o_jz, s_red);
    if (blockIdx.x == gridDim.x - 1) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Two cells of a row per thread, for 16-bit storage: the cells x and x + 1
// (x even) share one 32-bit word of every PDF plane they store, and their
// pulled values come from 32-bit words too: c_x = 0 from the pair's own word,
// c_x = -1 from its own and the right neighbour's, c_x = +1 from the left
// neighbour's and its own.  The collision runs on f32x2 instructions across the
// two cells (collide_cumulant_v or collide_srt_smag_v on float2), bit for bit
// the one-cell evaluation,
// and each store packs the pair with one conversion.  Half the threads of
// k_bulk, each with two cells' work and about half the instructions per cell;
// nx must be even (rows and planes then start on 32-bit words).  The launch's
// block is (tile_x / 2, tile_y).
template <typename T>
struct Pack16;
template <>
struct Pack16<__nv_bfloat16> {
    static __device__ __forceinline__ float lo(unsigned w) { return __uint_as_float(w << 16); }
    static __device__ __forceinline__ float hi(unsigned w) { return __uint_as_float(w & 0xFFFF0000u); }
    static __device__ __forceinline__ unsigned pack(float a, float b)
    {
        const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);  // a at the lower address
        return *reinterpret_cast<const unsigned*>(&v);
    }
};
template <>
struct Pack16<__half> {
    static __device__ __forceinline__ float lo(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu))); }
    static __device__ __forceinline__ float hi(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
    static __device__ __forceinline__ unsigned pack(float a, float b)
    {
        const __half2 v = __floats2half2_rn(a, b);
        return *reinterpret_cast<const unsigned*>(&v);
    }
};
__device__ __forceinline__ unsigned ld_word(const unsigned* p)
{
    unsigned v;
    asm("ld.global.nc.L2::256B.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

template <int COLL, typename T, bool DIAG, bool SINGLE>
__global__ void __launch_bounds__(128, COLL == COLL_CUMULANT ? 4 : 5) k_bulk2(const StepArgs A, const BulkParams P)
{
    static_assert(sizeof(T) == 2, "paired cells are for 16-bit storage");
    using W = Pack16<T>;
    __shared__ double s_red[DIAG ? 8 : 1][4];
    const unsigned long long tile = ld_tile(A.tiles + blockIdx.x);
    const int inst = SINGLE ? 0 : tile_lattice(tile);
    const LatHot& L = P.lat[inst];
    const int z = (int)((tile >> 32) & 0xFFFF);
    const int y = (int)((tile >> 16) & 0xFFFF) + threadIdx.y;
    const int x0 = (int)(tile & 0xFFFF);
    const int x = x0 + 2 * (int)threadIdx.x;  // cells x, x + 1
    const long long step = __ldcg(A.step_slot + A.parity);
    if (A.write_step && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        A.step_slot[A.parity ^ 1] = step + 1;
        A.diag_flag[A.parity ^ 1] = A.diag_every > 0 && (step + 1) % A.diag_every == 0;
    }
    double o_m = 0.0, o_jx = 0.0, o_jy = 0.0, o_jz = 0.0;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    if (x < nx && y < ny) {
        const unsigned* __restrict__ src = (const unsigned*)L.f[A.parity];
        unsigned* __restrict__ dst = (unsigned*)L.f[A.parity ^ 1];
        const unsigned N2 = L.N >> 1;  // words per plane
        int ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
        if (ym < 0) ym += ny; if (yp >= ny) yp -= ny;
        if (zm < 0) zm += nz; if (zp >= nz) zp -= nz;
        const unsigned ys[3] = {(unsigned)yp, (unsigned)y, (unsigned)ym};
        const unsigned zs[3] = {(unsigned)zp, (unsigned)z, (unsigned)zm};
        const unsigned nx2 = (unsigned)nx >> 1, nxy2 = nx2 * (unsigned)ny;
        const unsigned xw = (unsigned)x >> 1;
        float2 h[27];
        // words of the left pair (x - 2, x - 1) and right pair (x + 2, x + 3),
        // relative to the pair's own: in tiles clear of both x faces (uniform over
        // the CTA) -1 and +1; at the faces wrapped (periodic x) or, with an inlet
        // and outlet, the pair's own word (the inlet replaces the x = 0 cell's
        // c_x = +1 values below; at the outlet the last cell's c_x = -1 source is
        // the clamped cell x + 1 itself, the high half of its own word)
        int dl = -1, dr = 1;
        bool clamp_r = false;
        if (!(x0 > 0 && x0 + 2 * (int)blockDim.x < nx)) {
            if (x == 0) dl = L.inout ? 0 : (int)nx2 - 1;
            if (x + 2 == nx) {
                dr = L.inout ? 0 : -((int)nx2 - 1);
                clamp_r = L.inout != 0;
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const unsigned* zr = src + zs[k] * nxy2;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const unsigned* r = zr + (ys[j] * nx2 + xw);
                const int q = k * 9 + j * 3;
                const unsigned* p0 = r + (size_t)q * N2;         // c_x = -1: sources x + 1, x + 2
                const unsigned* p1 = r + (size_t)(q + 1) * N2;   // c_x = 0
                const unsigned* p2 = r + (size_t)(q + 2) * N2;   // c_x = +1: sources x - 1, x
                const unsigned o0 = ld_word(p0), r0 = ld_word(p0 + dr);
                const unsigned o1 = ld_word(p1);
                const unsigned l2 = ld_word(p2 + dl), o2 = ld_word(p2);
                h[q] = make_float2(W::hi(o0), clamp_r ? W::hi(r0) : W::lo(r0));
                h[q + 1] = make_float2(W::lo(o1), W::hi(o1));
                h[q + 2] = make_float2(W::hi(l2), W::lo(o2));
            }
        }
        if (L.inout && x == 0) {
            // the x = 0 cell's nine directions with c_x = +1 across the inlet face,
            // from the ghost columns (y - c_y, z - c_z); then this column's ghosts
            // for step n+1
            const DevDomain* D = A.dom + inst;
            const float* gb = D->inflow_ghost[step & 1];
            const int plane = ny * nz;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int j = 0; j < 3; ++j) h[k * 9 + j * 3 + 2].x = gb[(k * 3 + j) * plane + (int)zs[k] * ny + (int)ys[j]];
            write_inlet_ghost(D, step + 1, y, z);
        }
        float2 m, jx, jy, jz;
        if (COLL == COLL_CUMULANT)
            collide_cumulant_v<float2>(h, bc2(L.body[0]), bc2(L.body[1]), bc2(L.body[2]), L.omega, m, jx, jy, jz);
        else
            collide_srt_smag_v<float2>(h, bc2(L.body[0]), bc2(L.body[1]), bc2(L.body[2]), L.tau0, L.smag_c2, m, jx,
                                       jy, jz);
        if (DIAG) {
            o_m = (double)m.x + (double)m.y;
            o_jx = (double)jx.x + (double)jx.y;
            o_jy = (double)jy.x + (double)jy.y;
            o_jz = (double)jz.x + (double)jz.y;
        }
        unsigned* c = dst + (((unsigned)z * (unsigned)ny + (unsigned)y) * nx2 + xw);
#pragma unroll
        for (int q = 0; q < 27; ++q) c[(size_t)q * N2] = W::pack(h[q].x, h[q].y);
    }
    if (DIAG) diag_close(A, A.dom + inst, step, o_m, o_jx, o_jy, o_jz, s_red);
    if (blockIdx.x == gridDim.x - 1) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------------ in-place (AA) step

// The in-place scheme keeps one PDF array A.  Before every even step it holds
// the pull scheme's state, A[q][x] = f*_q(x) of the last collision.  A step
// reads for each cell and direction q one "source" and, on even steps, writes
// the post-collision f*_q into the source it read for the opposite direction
// qbar; odd steps read A[qbar][x] and write A[q][x].  A source is the slot the
// pull rules of load_cell / boundary_patch name (the pull source, the
// cell's own opposite slot at a no-slip face, the mirrored slot at a free-slip
// face), or a value no slot holds: an inlet ghost population, or at the
// outlet the zero-gradient copy of the last plane, which the in-place scheme
// keeps in its own buffer (the slot the pull scheme reads there has another
// reader, who overwrites it).  Every slot has one reader per step, so each
// slot is read and then written by one thread, and after every odd step the
// array is the pull scheme's state again, value for value.
struct AaSource {
    unsigned off;  // slot offset (slot true)
    float val;     // the value otherwise
    bool slot;
};

// The source of direction q at cell (x, y, z) on the step `step`, by the pull
// rules in their order: no-slip, free-slip, periodic wrap, x inlet / outlet.
__device__ __forceinline__ AaSource aa_source(const DevDomain* D, int q, int x, int y, int z, long long step)
{
    const int n[3] = {D->nx, D->ny, D->nz};
    const int p[3] = {x, y, z};
    const int c[3] = {qcx(q), qcy(q), qcz(q)};
    const unsigned N = (unsigned)D->N;
    AaSource r;
    r.off = 0u;
    r.val = 0.0f;
    r.slot = true;
    int s[3], cm[3];
    bool wall = false;
    for (int a = 0; a < 3; ++a) {
        s[a] = p[a] - c[a];
        cm[a] = c[a];
        if (D->bc[a] == BC_NOSLIP && (s[a] < 0 || s[a] >= n[a])) wall = true;
    }
    if (wall) {
        r.off = (unsigned)(26 - q) * N + (((unsigned)z * (unsigned)n[1] + (unsigned)y) * (unsigned)n[0] + (unsigned)x);
        return r;
    }
    for (int a = 0; a < 3; ++a)
        if (D->bc[a] == BC_FREESLIP && (s[a] < 0 || s[a] >= n[a])) {
            cm[a] = -c[a];
            s[a] = p[a];
        }
    for (int a = 0; a < 3; ++a)
        if (D->bc[a] == BC_PERIODIC) s[a] = s[a] < 0 ? s[a] + n[a] : (s[a] >= n[a] ? s[a] - n[a] : s[a]);
    if (D->bc[0] == BC_INOUT && (s[0] < 0 || s[0] >= n[0])) {
        // ghost of the inlet (c_x = +1) or the outlet copy of the last plane (c_x = -1)
        const float* buf = s[0] < 0 ? D->inflow_ghost[step & 1] : D->outlet[step & 1];
        r.val = buf[((cm[2] + 1) * 3 + (cm[1] + 1)) * (n[1] * n[2]) + s[2] * n[1] + s[1]];
        r.slot = false;
        return r;
    }
    const int qm = (cm[2] + 1) * 9 + (cm[1] + 1) * 3 + (cm[0] + 1);
    r.off = (unsigned)qm * N + (((unsigned)s[2] * (unsigned)n[1] + (unsigned)s[1]) * (unsigned)n[0] + (unsigned)s[0]);
    return r;
}

// Neighbour rows and columns of cell (x, y, z) away from the wall faces:
// source coordinates for c = -1, 0, +1 (wrapped on periodic axes, clamped at
// the x inlet and outlet, whose cells replace those values), and whether the
// cell lies on a no-slip or free-slip face.
struct AaNbr {
    unsigned xs[3], ys[3], zs[3];
    bool face;
};
__device__ __forceinline__ AaNbr aa_neighbours(const DevDomain* D, int x, int y, int z)
{
    const int nx = D->nx, ny = D->ny, nz = D->nz;
    int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
    AaNbr r;
    r.face = false;
    if (D->bc[0] == BC_PERIODIC) { if (xm < 0) xm += nx; if (xp >= nx) xp -= nx; }
    else if (D->bc[0] == BC_INOUT) { xm = max(xm, 0); xp = min(xp, nx - 1); }
    else { r.face = r.face || x == 0 || x == nx - 1; }
    if (D->bc[1] == BC_PERIODIC) { if (ym < 0) ym += ny; if (yp >= ny) yp -= ny; }
    else { r.face = r.face || y == 0 || y == ny - 1; }
    if (D->bc[2] == BC_PERIODIC) { if (zm < 0) zm += nz; if (zp >= nz) zp -= nz; }
    else { r.face = r.face || z == 0 || z == nz - 1; }
    r.xs[0] = (unsigned)xp; r.xs[1] = (unsigned)x; r.xs[2] = (unsigned)xm;
    r.ys[0] = (unsigned)yp; r.ys[1] = (unsigned)y; r.ys[2] = (unsigned)ym;
    r.zs[0] = (unsigned)zp; r.zs[1] = (unsigned)z; r.zs[2] = (unsigned)zm;
    return r;
}
__device__ __forceinline__ unsigned aa_row(const AaNbr& nb, int k, int j, int ny, int nx)
{
    return (nb.zs[k] * (unsigned)ny + nb.ys[j]) * (unsigned)nx;
}

// The in-place update of a cell on a no-slip or free-slip face, out of line
// (few cells take it, and the direct path then needs no stack): every source
// by the pull rules (aa_source), the inlet ghost for step n+1, the outlet copy.
// Returns (mass, momentum) of the cell for the diagnostic sums.
template <int COLL, typename T, bool ODD, bool ROTOR>
__device__ __noinline__ float4 aa_face_cell(const DevDomain* D, int x, int y, int z, long long step, int n_cull,
                                            const float4* s_pos, const float4* s_frc, const int* s_tag)
{
    T* f = (T*)D->f[0];
    const unsigned uN = (unsigned)D->N;
    const int nx = D->nx, ny = D->ny;
    const unsigned cell = ((unsigned)z * (unsigned)ny + (unsigned)y) * (unsigned)nx + (unsigned)x;
    float h[27];
    for (int q = 0; q < 27; ++q) {
        const AaSource S = aa_source(D, q, x, y, z, step);
        // odd steps read A[qbar][x] wherever the even rule names a slot
        h[q] = !S.slot ? S.val : Io<T>::ldw(f + (ODD ? (unsigned)(26 - q) * uN + cell : S.off));
    }
    const bool inout = D->bc[0] == BC_INOUT;
    if (inout && x == 0) write_inlet_ghost(D, step + 1, y, z);
    float F[3] = {D->body[0], D->body[1], D->body[2]};
    if (ROTOR) rotor_force(D, step, x, y, z, n_cull, s_pos, s_frc, s_tag, F);
    float m, jx, jy, jz;
    if (COLL == COLL_CUMULANT)
        collide_cumulant(h, F[0], F[1], F[2], D->omega, m, jx, jy, jz);
    else
        collide_srt_smag(h, F[0], F[1], F[2], D->tau0, D->smag_c2, m, jx, jy, jz);
    if (inout && x == nx - 1) {
        float* ob = D->outlet[(step + 1) & 1];
        const int plane = ny * D->nz, col = z * ny + y;
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) ob[(k * 3 + j) * plane + col] = Io<T>::round(h[k * 9 + j * 3]);
    }
    for (int q = 0; q < 27; ++q) {
        if (ODD) {
            Io<T>::st(f + ((unsigned)q * uN + cell), h[q]);
        } else {
            const AaSource S = aa_source(D, 26 - q, x, y, z, step);  // the slot read for the opposite direction
            if (S.slot) Io<T>::st(f + S.off, h[q]);                  // else f*_q leaves the lattice
        }
    }
    return make_float4(m, jx, jy, jz);
}

// The in-place update of one cell (x, y, z), for the bulk and the rotor
// launches.  ROTOR: the cell lies in a rotor tile and adds the regularised
// blade force.  Returns the cell's mass and momentum contributions.  Cells on
// a wall face take aa_face_cell; the x inlet and outlet cells stay on the
// direct path: the nine directions that cross the face are read from the
// inlet ghosts or the outlet copy, and the nine post-collision values that
// leave through it are not stored.
template <int COLL, typename T, bool ODD, bool ROTOR>
__device__ __forceinline__ void aa_cell(const DevDomain* D, int x, int y, int z, long long step, int n_cull,
                                        const float4* s_pos, const float4* s_frc, const int* s_tag, float& m, float& jx,
                                        float& jy, float& jz)
{
    T* f = (T*)D->f[0];
    const unsigned uN = (unsigned)D->N;
    const int nx = D->nx, ny = D->ny;
    const bool inout = D->bc[0] == BC_INOUT;
    float h[27];
    {
        const AaNbr nb = aa_neighbours(D, x, y, z);
        if (nb.face) {
            const float4 r = aa_face_cell<COLL, T, ODD, ROTOR>(D, x, y, z, step, n_cull, s_pos, s_frc, s_tag);
            m = r.x;
            jx = r.y;
            jy = r.z;
            jz = r.w;
            return;
        }
        if (ODD) {
            const unsigned cell = ((unsigned)z * (unsigned)ny + (unsigned)y) * (unsigned)nx + (unsigned)x;
#pragma unroll
            for (int q = 0; q < 27; ++q) h[q] = Io<T>::ldw(f + ((unsigned)(26 - q) * uN + cell));
        } else {
#pragma unroll
            for (int q = 0; q < 27; ++q)
                h[q] = Io<T>::ldw(f + ((unsigned)q * uN + aa_row(nb, q / 9, (q / 3) % 3, ny, nx) + nb.xs[q % 3]));
        }
        if (inout && (x == 0 || x == nx - 1)) {
            // across the inlet: ghosts of the columns (y - c_y, z - c_z); across the
            // outlet: the last plane's copies there (zero-gradient)
            // (two branches: a run-time index into h would put h in local memory)
            const int plane = ny * D->nz;
            if (x == 0) {
                const float* gb = D->inflow_ghost[step & 1];
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        h[k * 9 + j * 3 + 2] = gb[(k * 3 + j) * plane + (int)nb.zs[k] * ny + (int)nb.ys[j]];
            } else {
                const float* ob = D->outlet[step & 1];
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        h[k * 9 + j * 3] = ob[(k * 3 + j) * plane + (int)nb.zs[k] * ny + (int)nb.ys[j]];
            }
        }
    }
    if (inout && x == 0) write_inlet_ghost(D, step + 1, y, z);
    float F[3] = {D->body[0], D->body[1], D->body[2]};
    if (ROTOR) rotor_force(D, step, x, y, z, n_cull, s_pos, s_frc, s_tag, F);
    if (COLL == COLL_CUMULANT)
        collide_cumulant(h, F[0], F[1], F[2], D->omega, m, jx, jy, jz);
    else
        collide_srt_smag(h, F[0], F[1], F[2], D->tau0, D->smag_c2, m, jx, jy, jz);
    if (inout && x == nx - 1) {
        // the outlet copy for step n+1: f*_q of the last plane, directions with
        // c_x = -1, as the array would hold it (rounded to the storage type)
        float* ob = D->outlet[(step + 1) & 1];
        const int plane = ny * D->nz, col = z * ny + y;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) ob[(k * 3 + j) * plane + col] = Io<T>::round(h[k * 9 + j * 3]);
    }
    // the store slots are the load slots, recomputed from opaque copies of
    // the inputs: kept live across the collision they would spill
    unsigned long long fa = (unsigned long long)f;
    int xo = x, yo = y, zo = z;
    asm volatile("" : "+l"(fa), "+r"(xo), "+r"(yo), "+r"(zo));
    f = (T*)fa;
    if (ODD) {
        const unsigned cell = ((unsigned)zo * (unsigned)ny + (unsigned)yo) * (unsigned)nx + (unsigned)xo;
#pragma unroll
        for (int q = 0; q < 27; ++q) Io<T>::st(f + ((unsigned)q * uN + cell), h[q]);
    } else {
        const AaNbr nb = aa_neighbours(D, xo, yo, zo);
        const bool at_in = inout && xo == 0, at_out = inout && xo == nx - 1;
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            // f*_q goes to the slot read for the opposite direction, unless it
            // leaves through the inlet or the outlet
            if ((qcx(q) == -1 && at_in) || (qcx(q) == 1 && at_out)) continue;
            const int p = 26 - q;
            Io<T>::st(f + ((unsigned)p * uN + aa_row(nb, p / 9, (p / 3) % 3, ny, nx) + nb.xs[p % 3]), h[q]);
        }
    }
}

// The time step on a single PDF array (the AA pattern), as launches like
// k_step: ROTOR over the rotor tiles (element culling, force gather; the
// actuator line of the next step follows as its own launch, whose sampling
// reads the array in the layout this step leaves), then the rest, which may
// overlap them.  Rotor tiles cover up to kRotorPlanes planes, one
// after the other; bulk tiles one plane.
template <int COLL, typename T, bool ODD, bool ROTOR>
__global__ void __launch_bounds__(256, ROTOR ? 2 : (COLL == COLL_CUMULANT ? 4 : 3)) k_step_aa(const StepArgs A)
{
    if (ROTOR) asm volatile("griddepcontrol.launch_dependents;");
    constexpr int kCull = 128;
    __shared__ double s_red[8][4];
    __shared__ float4 s_pos[ROTOR ? kCull : 1], s_frc[ROTOR ? kCull : 1];
    __shared__ int s_tag[ROTOR ? kCull : 1];
    __shared__ int s_cnt[8];
    const unsigned long long tile = ld_tile(A.tiles + blockIdx.x);
    const int z0 = (int)((tile >> 32) & 0xFFFF);
    const int y = (int)((tile >> 16) & 0xFFFF) + threadIdx.y;
    const int x = (int)(tile & 0xFFFF) + threadIdx.x;
    const DevDomain* D = A.dom + tile_lattice(tile);
    const long long step = __ldcg(A.step_slot + A.parity);
    if (A.write_step && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        A.step_slot[A.parity ^ 1] = step + 1;
        A.diag_flag[A.parity ^ 1] = A.diag_every > 0 && (step + 1) % A.diag_every == 0;
    }
    const bool diag = __ldcg(A.diag_flag + A.parity) != 0;
    using Acc = typename std::conditional<ROTOR, double, float>::type;
    Acc o_m = 0, o_jx = 0, o_jy = 0, o_jz = 0;
    if constexpr (ROTOR) {
        const int planes = tile_planes(tile);
        const int z1 = min(z0 + planes, D->nz);
        const int n_cull = cull_rotor_elements<kCull>(D, tile, step, z0, z1, s_pos, s_frc, s_tag, s_cnt);
        if (x < D->nx && y < D->ny) {
#pragma unroll 1
            for (int z = z0; z < z1; ++z) {
                float m, jx, jy, jz;
                aa_cell<COLL, T, ODD, true>(D, x, y, z, step, n_cull, s_pos, s_frc, s_tag, m, jx, jy, jz);
                if (diag) {
                    o_m += m;
                    o_jx += jx;
                    o_jy += jy;
                    o_jz += jz;
                }
            }
        }
    } else {
        if (x < D->nx && y < D->ny) {
            float m, jx, jy, jz;
            aa_cell<COLL, T, ODD, false>(D, x, y, z0, step, -1, nullptr, nullptr, nullptr, m, jx, jy, jz);
            if (diag) {
                o_m = m;
                o_jx = jx;
                o_jy = jy;
                o_jz = jz;
            }
        }
    }
    if (diag) diag_close(A, D, step, (double)o_m, (double)o_jx, (double)o_jy, (double)o_jz, s_red);
    if constexpr (!ROTOR) {
        if (blockIdx.x == gridDim.x - 1) asm volatile("griddepcontrol.wait;" ::: "memory");
    }
}

// Outlet copies of the last plane for step `step` from the array's current
// (pull-scheme) state, after a state change of an in-place lattice.
// The in-place step over the tiles without a no-slip or free-slip face cell,
// two cells of a row per thread (16-bit storage, nx even), as k_bulk2 does for
// the pull scheme.  Odd steps read a cell's own opposite slots and write its own
// slots: for the pair (x, x + 1) one 32-bit word per plane each way.  Even steps
// pull from the neighbours' words like k_bulk2 and store f*_q into the slot read
// for the opposite direction: with no x shift that is one word of the pair's
// own; shifted by one cell it straddles two words, and the two cells store their
// halves with 16-bit stores.  Every slot a thread writes is one it read itself;
// a neighbour may rewrite the other half of a word this thread loaded, a half it
// does not use.  Inlet and outlet as in aa_cell.  Bit for bit the one-cell form.
__device__ __forceinline__ void st_half(void* p, unsigned short v)
{
    asm volatile("st.global.b16 [%0], %1;" ::"l"(p), "h"(v) : "memory");
}
template <typename T>
__device__ __forceinline__ unsigned short to_bits16(float v);
template <>
__device__ __forceinline__ unsigned short to_bits16<__nv_bfloat16>(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <>
__device__ __forceinline__ unsigned short to_bits16<__half>(float v)
{
    return __half_as_ushort(__float2half_rn(v));
}

template <int COLL, typename T, bool ODD, bool SINGLE>
__global__ void __launch_bounds__(128, SINGLE ? 5 : 4) k_step_aa2(const StepArgs A, const BulkParams P)
{
    static_assert(sizeof(T) == 2, "paired cells are for 16-bit storage");
    using W = Pack16<T>;
    __shared__ double s_red[8][4];
    const unsigned long long tile = ld_tile(A.tiles + blockIdx.x);
    const int inst = SINGLE ? 0 : tile_lattice(tile);
    const LatHot& L = P.lat[inst];
    const int z = (int)((tile >> 32) & 0xFFFF);
    const int y = (int)((tile >> 16) & 0xFFFF) + threadIdx.y;
    const int x0 = (int)(tile & 0xFFFF);
    const int x = x0 + 2 * (int)threadIdx.x;  // cells x, x + 1
    const DevDomain* D = A.dom + inst;  // the inlet and outlet buffers only
    const long long step = __ldcg(A.step_slot + A.parity);
    if (A.write_step && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        A.step_slot[A.parity ^ 1] = step + 1;
        A.diag_flag[A.parity ^ 1] = A.diag_every > 0 && (step + 1) % A.diag_every == 0;
    }
    const bool diag = __ldcg(A.diag_flag + A.parity) != 0;
    double o_m = 0.0, o_jx = 0.0, o_jy = 0.0, o_jz = 0.0;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    if (x < nx && y < ny) {
        unsigned* fw = (unsigned*)L.f[0];
        const unsigned N2 = L.N >> 1;  // words per plane
        const bool inout = L.inout != 0;
        int ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
        if (ym < 0) ym += ny; if (yp >= ny) yp -= ny;
        if (zm < 0) zm += nz; if (zp >= nz) zp -= nz;
        const unsigned ys[3] = {(unsigned)yp, (unsigned)y, (unsigned)ym};
        const unsigned zs[3] = {(unsigned)zp, (unsigned)z, (unsigned)zm};
        const unsigned nx2 = (unsigned)nx >> 1, nxy2 = nx2 * (unsigned)ny;
        const unsigned xw = (unsigned)x >> 1;
        const bool at_in = inout && x == 0, at_out = inout && x + 2 == nx;
        // left and right neighbour words relative to the pair's own: wrapped on a
        // periodic x, else the own word (the inlet and outlet replace those values)
        int dl = -1, dr = 1;
        if (x == 0) dl = inout ? 0 : (int)nx2 - 1;
        if (x + 2 == nx) dr = inout ? 0 : -((int)nx2 - 1);
        float2 h[27];
        if (ODD) {
            const unsigned* own = fw + (((unsigned)z * (unsigned)ny + (unsigned)y) * nx2 + xw);
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const unsigned w = own[(size_t)(26 - q) * N2];
                h[q] = make_float2(W::lo(w), W::hi(w));
            }
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const unsigned* zr = fw + zs[k] * nxy2;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const unsigned* r = zr + (ys[j] * nx2 + xw);
                    const int q = k * 9 + j * 3;
                    const unsigned* p0 = r + (size_t)q * N2;         // c_x = -1: sources x + 1, x + 2
                    const unsigned* p1 = r + (size_t)(q + 1) * N2;   // c_x = 0
                    const unsigned* p2 = r + (size_t)(q + 2) * N2;   // c_x = +1: sources x - 1, x
                    const unsigned o0 = *p0, r0 = p0[dr];
                    const unsigned o1 = *p1;
                    const unsigned l2 = p2[dl], o2 = *p2;
                    h[q] = make_float2(W::hi(o0), W::lo(r0));
                    h[q + 1] = make_float2(W::lo(o1), W::hi(o1));
                    h[q + 2] = make_float2(W::hi(l2), W::lo(o2));
                }
            }
        }
        const int plane = ny * nz;
        if (at_in) {
            // the x = 0 cell across the inlet: ghosts of the columns (y - c_y, z - c_z)
            const float* gb = D->inflow_ghost[step & 1];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    h[k * 9 + j * 3 + 2].x = gb[(k * 3 + j) * plane + (int)zs[k] * ny + (int)ys[j]];
        }
        if (at_out) {
            // the x = nx - 1 cell across the outlet: the last plane's copies there
            const float* ob = D->outlet[step & 1];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    h[k * 9 + j * 3].y = ob[(k * 3 + j) * plane + (int)zs[k] * ny + (int)ys[j]];
        }
        if (at_in) write_inlet_ghost(D, step + 1, y, z);
        float2 m, jx, jy, jz;
        if (COLL == COLL_CUMULANT)
            collide_cumulant_v<float2>(h, bc2(L.body[0]), bc2(L.body[1]), bc2(L.body[2]), L.omega, m, jx, jy, jz);
        else
            collide_srt_smag_v<float2>(h, bc2(L.body[0]), bc2(L.body[1]), bc2(L.body[2]), L.tau0, L.smag_c2, m, jx,
                                       jy, jz);
        if (diag) {
            o_m = (double)m.x + (double)m.y;
            o_jx = (double)jx.x + (double)jx.y;
            o_jy = (double)jy.x + (double)jy.y;
            o_jz = (double)jz.x + (double)jz.y;
        }
        if (at_out) {
            // the outlet copy for step n+1: f*_q of the last plane, directions with
            // c_x = -1, as the array would hold it (rounded to the storage type)
            float* ob = D->outlet[(step + 1) & 1];
            const int col = z * ny + y;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int j = 0; j < 3; ++j) ob[(k * 3 + j) * plane + col] = Io<T>::round(h[k * 9 + j * 3].y);
        }
        // the store slots are the load slots, recomputed from opaque copies of the
        // coordinates: kept live across the collision they would spill
        unsigned long long fa = (unsigned long long)fw;
        int xo = x, yo = y, zo = z;
        asm volatile("" : "+l"(fa), "+r"(xo), "+r"(yo), "+r"(zo));
        unsigned* fs = (unsigned*)fa;
        const unsigned xwo = (unsigned)xo >> 1;
        if (ODD) {
            unsigned* own = fs + (((unsigned)zo * (unsigned)ny + (unsigned)yo) * nx2 + xwo);
#pragma unroll
            for (int q = 0; q < 27; ++q) own[(size_t)q * N2] = W::pack(h[q].x, h[q].y);
        } else {
            int ymo = yo - 1, ypo = yo + 1, zmo = zo - 1, zpo = zo + 1;
            if (ymo < 0) ymo += ny; if (ypo >= ny) ypo -= ny;
            if (zmo < 0) zmo += nz; if (zpo >= nz) zpo -= nz;
            const unsigned yso[3] = {(unsigned)ypo, (unsigned)yo, (unsigned)ymo};
            const unsigned zso[3] = {(unsigned)zpo, (unsigned)zo, (unsigned)zmo};
            const bool in_o = inout && xo == 0, out_o = inout && xo + 2 == nx;
            int dlo = -1, dro = 1;
            if (xo == 0) dlo = inout ? 0 : (int)nx2 - 1;
            if (xo + 2 == nx) dro = inout ? 0 : -((int)nx2 - 1);
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                // f*_q goes to the slot read for the opposite direction p, in plane p
                // at the cells x + c_q, unless it leaves through the inlet or the outlet
                const int p = 26 - q;
                unsigned* w = fs + (size_t)p * N2 + zso[p / 9] * nxy2 + yso[(p / 3) % 3] * nx2 + xwo;
                if (qcx(q) == 0) {
                    *w = W::pack(h[q].x, h[q].y);
                } else if (qcx(q) == 1) {  // cells x + 1 (high half of the own word) and x + 2
                    *((unsigned short*)w + 1) = to_bits16<T>(h[q].x);
                    if (!out_o) *(unsigned short*)(w + dro) = to_bits16<T>(h[q].y);
                } else {                   // cells x - 1 (high half of the left word) and x
                    if (!in_o) *((unsigned short*)(w + dlo) + 1) = to_bits16<T>(h[q].x);
                    *(unsigned short*)w = to_bits16<T>(h[q].y);
                }
            }
        }
    }
    if (diag) diag_close(A, D, step, o_m, o_jx, o_jy, o_jz, s_red);
    if (blockIdx.x == gridDim.x - 1) asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename T>
__global__ void k_outlet_fill(const DevDomain* D, long long step)
{
    const int plane = D->ny * D->nz;
    const T* f = (const T*)D->f[0];
    float* ob = D->outlet[step & 1];
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < plane; col += gridDim.x * blockDim.x) {
        const int y = col % D->ny, z = col / D->ny;
        const long long cell = ((long long)z * D->ny + y) * D->nx + (D->nx - 1);
        for (int g = 0; g < 9; ++g) ob[g * plane + col] = Io<T>::ldcg(f + (size_t)(g * 3) * D->N + cell);
    }
}

// ------------------------------------------------------------------ staged step (TMA bulk copies)

// Elements per 16-byte chunk: the halo kept on each side of a staged row.
template <typename T> __host__ __device__ constexpr int halo_of() { return 16 / (int)sizeof(T); }

// Stages of the shared-memory ring for a segment width: four while a stage
// (27 rows of W + 2H elements) is at most 16 KB, else three.
__host__ __device__ inline int bulk_stages(int width, int elem_bytes)
{
    const int stage = 27 * (width + 2 * (16 / elem_bytes)) * elem_bytes;
    return stage <= 16384 ? 4 : 3;
}
__host__ __device__ inline size_t bulk_smem_bytes(int width, int elem_bytes)
{
    return (size_t)bulk_stages(width, elem_bytes) * 27 * (width + 2 * (16 / elem_bytes)) * elem_bytes;
}

constexpr int kMaxStages = 4;
constexpr long long kWaitCycles = kDefaultWaitCycles;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// Bounded wait for the phase of the given parity: tries until `limit` SM clock
// cycles have passed, false if the phase did not complete by then (a limit of
// 0 gives up before the first try).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit)
{
    const unsigned a = smem_addr(bar);
    const long long t0 = clock64();
    for (;;) {
        if (clock64() - t0 >= limit) return false;
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
}
// One row of bytes (16-byte aligned, multiple of 16) from global to shared memory,
// completing on the barrier's transaction count.
__device__ __forceinline__ void bulk_row(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Issue the 27 row copies of work-list entry `it` (a row segment, tile_y = 1)
// into `stage`: lane q copies direction q's source row (y - c_y, z - c_z),
// wrapped or clamped as in load_cell, elements [x0 - H, x0 + W + H) clipped to
// the row, to stage[q][x - x0 + H].  nx is a multiple of H, so the copy starts
// and ends on 16-byte boundaries.  Warp-wide; lane 0 arms the barrier.
template <typename T>
__device__ __forceinline__ void bulk_issue(const StepArgs& A, unsigned it, T* stage, unsigned long long* bar, int W)
{
    constexpr int H = halo_of<T>();
    const int lane = threadIdx.x & 31;
    const unsigned long long tile = A.tiles[it];
    const DevDomain* D = A.dom + tile_lattice(tile);
    const int z = (int)((tile >> 32) & 0xFFFF), y = (int)((tile >> 16) & 0xFFFF), x0 = (int)(tile & 0xFFFF);
    const int nx = D->nx, ny = D->ny, nz = D->nz;
    const int lo = max(x0 - H, 0), hi = min(x0 + W + H, nx);
    const unsigned bytes = (unsigned)(hi - lo) * (unsigned)sizeof(T);
    if (lane == 0) mbar_expect_tx(bar, 27u * bytes);
    __syncwarp();
    if (lane < 27) {
        const int q = lane;
        int ys = y - ((q / 3) % 3 - 1), zs = z - (q / 9 - 1);
        const int by = D->bc[1], bz = D->bc[2];
        if (ys < 0) ys = by == BC_PERIODIC ? ys + ny : 0;
        if (ys >= ny) ys = by == BC_PERIODIC ? ys - ny : ny - 1;
        if (zs < 0) zs = bz == BC_PERIODIC ? zs + nz : 0;
        if (zs >= nz) zs = bz == BC_PERIODIC ? zs - nz : nz - 1;
        const T* row = (const T*)D->f[A.parity] + ((unsigned)q * (unsigned)D->N + ((unsigned)zs * ny + ys) * (unsigned)nx);
        bulk_row(stage + q * (W + 2 * H) + (lo - x0 + H), row + lo, bytes, bar);
    }
}

// k_step with the source rows staged in shared memory by TMA bulk copies:
// persistent CTAs walk the work list (one row segment of blockDim.x cells per
// entry) through a ring of 3-4 stages, so two or three segments are in flight
// while one collides and the loads in flight hold no registers.  Same
// arithmetic, same results as k_step.  Every barrier wait is bounded: a wait
// that gives up sets ERR_TIMEOUT, and the CTA waits (bounded) for its copies in
// flight before it returns.
template <int COLL, typename T>
__global__ void __launch_bounds__(256, 3) k_step_staged(const StepArgs A)
{
    constexpr int H = halo_of<T>();
    constexpr int kCull = 128;
    extern __shared__ __align__(128) unsigned char stage_raw[];
    __shared__ __align__(8) unsigned long long s_full[kMaxStages];
    __shared__ double s_red[8][4];
    __shared__ int s_abort;
    __shared__ float4 s_pos[kCull], s_frc[kCull];
    __shared__ int s_tag[kCull];
    __shared__ int s_cnt[8];
    const int W = blockDim.x;
    const int rowlen = W + 2 * H;
    const int S = bulk_stages(W, (int)sizeof(T));
    T* const stage0 = (T*)stage_raw;
    const int tid = threadIdx.x;
    const int par = A.parity;
    const long long step = __ldcg(A.step_slot + par);
    if (blockIdx.x == 0 && tid == 0) {
        A.step_slot[par ^ 1] = step + 1;
        A.diag_flag[par ^ 1] = A.diag_every > 0 && (step + 1) % A.diag_every == 0;
    }
    const bool diag = __ldcg(A.diag_flag + par) != 0;
    float o_m = 0.0f, o_jx = 0.0f, o_jy = 0.0f, o_jz = 0.0f;
    const unsigned G = gridDim.x;
    // segments of this CTA: blockIdx.x + k G, k = 0, 1, ...
    const unsigned n_mine = blockIdx.x < A.n_tiles ? (A.n_tiles - blockIdx.x + G - 1) / G : 0u;

    if (tid == 0) {
        for (int i = 0; i < S; ++i) mbar_init(s_full + i, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // prologue: the first S - 1 segments
    if (tid < 32)
        for (unsigned k = 0; k < (unsigned)(S - 1) && k < n_mine; ++k)
            bulk_issue<T>(A, blockIdx.x + k * G, stage0 + (size_t)k * 27 * rowlen, s_full + k, W);
    unsigned issued = min((unsigned)(S - 1), n_mine);
    unsigned k = 0;  // segments waited for

    for (; k < n_mine; ++k) {
        const unsigned it = blockIdx.x + k * G;
        // every thread is done with segment k - 1, whose stage the next copy reuses
        __syncthreads();
        if (s_abort) break;
        if (issued < n_mine) {
            if (tid < 32) {
                if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                bulk_issue<T>(A, blockIdx.x + issued * G, stage0 + (size_t)(issued % S) * 27 * rowlen,
                              s_full + issued % S, W);
            }
            ++issued;
        }
        const int sidx = (int)(k % S);
        if (!mbar_wait(s_full + sidx, (k / S) & 1u, A.wait_cycles)) {
            s_abort = 1;
            atomicOr(A.dom->err, ERR_TIMEOUT);
        }
        __syncthreads();
        if (s_abort) break;
        const T* st = stage0 + (size_t)sidx * 27 * rowlen;

        const unsigned long long tile = A.tiles[it];
        const bool rotor_tile = (tile >> 63) != 0;
        const DevDomain* D = A.dom + tile_lattice(tile);
        const int z = (int)((tile >> 32) & 0xFFFF);
        const int y = (int)((tile >> 16) & 0xFFFF);
        const int x0 = (int)(tile & 0xFFFF);
        const int x = x0 + tid;
        const int nx = D->nx, ny = D->ny, nz = D->nz;
        const unsigned uN = (unsigned)D->N;
        const T* __restrict__ src = (const T*)D->f[par];
        T* __restrict__ dst = (T*)D->f[par ^ 1];
        // rotor segment: cull the blade elements reaching it
        int n_cull = -1;
        if (rotor_tile) {
            const float tx0 = (float)x0, tx1 = (float)(x0 + W - 1), fy = (float)y, fz = (float)z;
            const float4* P = D->el_pos[step & 1];
            const float4* Fe = D->el_force[step & 1];
            const int lane = tid & 31, warp = tid >> 5, nwarps = W >> 5;
            int total = 0;
            for (int base = 0; base < D->n_el; base += W) {
                const int e = base + tid;
                bool keep = false;
                float4 pe = make_float4(0.f, 0.f, 0.f, 0.f);
                int t = 0;
                if (e < D->n_el) {
                    pe = __ldg(P + e);
                    while (t + 1 < D->n_turb && D->turb[t + 1].el_offset <= e) ++t;
                    const float cut = D->turb[t].cut;
                    keep = pe.x + cut >= tx0 && pe.x - cut <= tx1 && fabsf(pe.y - fy) <= cut && fabsf(pe.z - fz) <= cut;
                }
                const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
                if (lane == 0) s_cnt[warp] = __popc(m);
                __syncthreads();
                int off = total, chunk = 0;
                for (int w = 0; w < nwarps; ++w) {
                    if (w < warp) off += s_cnt[w];
                    chunk += s_cnt[w];
                }
                const int pos = off + __popc(m & ((1u << lane) - 1u));
                if (keep && pos < kCull) {
                    s_pos[pos] = pe;
                    s_frc[pos] = __ldg(Fe + e);
                    s_tag[pos] = t;
                }
                total += chunk;
                __syncthreads();
            }
            n_cull = total <= kCull ? total : -1;
        }
        if (x < nx) {
            float h[27];
            const int bx = D->bc[0], by = D->bc[1], bz = D->bc[2];
            // staged rows: x - c_x at column tid + H - c_x; periodic x wraps past the row ends (direct loads)
            const bool wrap_lo = bx == BC_PERIODIC && x == 0, wrap_hi = bx == BC_PERIODIC && x == nx - 1;
            const int cm = (x == 0) ? tid + H : tid + H - 1;          // source x - 1 (clamped at 0)
            const int cp = (x == nx - 1) ? tid + H : tid + H + 1;     // source x + 1 (clamped at nx - 1)
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const int cxq = q % 3 - 1;
                const int col = cxq == 1 ? cm : (cxq == 0 ? tid + H : cp);
                h[q] = to_float(st[q * rowlen + col]);
            }
            if (wrap_lo || wrap_hi) {
                int ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
                if (by == BC_PERIODIC) { if (ym < 0) ym += ny; if (yp >= ny) yp -= ny; }
                else { ym = max(ym, 0); yp = min(yp, ny - 1); }
                if (bz == BC_PERIODIC) { if (zm < 0) zm += nz; if (zp >= nz) zp -= nz; }
                else { zm = max(zm, 0); zp = min(zp, nz - 1); }
                const unsigned ys3[3] = {(unsigned)yp, (unsigned)y, (unsigned)ym};
                const unsigned zs3[3] = {(unsigned)zp, (unsigned)z, (unsigned)zm};
                const unsigned xw = wrap_lo ? (unsigned)(nx - 1) : 0u;
                const int cw = wrap_lo ? 2 : 0;  // the c_x that reads across the wrap
#pragma unroll
                for (int q = 0; q < 27; ++q) {
                    if (q % 3 != cw) continue;
                    const unsigned row = (zs3[q / 9] * (unsigned)ny + ys3[(q / 3) % 3]) * (unsigned)nx;
                    h[q] = Io<T>::ld(src + ((unsigned)q * uN + row + xw));
                }
            }
            // inlet and wall rules as in load_cell
            if (bx == BC_INOUT && x == 0) {
                int ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
                if (by == BC_PERIODIC) { if (ym < 0) ym += ny; if (yp >= ny) yp -= ny; }
                else { ym = max(ym, 0); yp = min(yp, ny - 1); }
                if (bz == BC_PERIODIC) { if (zm < 0) zm += nz; if (zp >= nz) zp -= nz; }
                else { zm = max(zm, 0); zp = min(zp, nz - 1); }
                const int ys3[3] = {yp, y, ym}, zs3[3] = {zp, z, zm};
                const float* gb = D->inflow_ghost[step & 1];
                const int plane = ny * nz;
#pragma unroll
                for (int kk = 0; kk < 3; ++kk)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int q = kk * 9 + j * 3 + 2;
                        const bool wall = (by == BC_NOSLIP && ((j == 2 && y == 0) || (j == 0 && y == ny - 1))) ||
                                          (bz == BC_NOSLIP && ((kk == 2 && z == 0) || (kk == 0 && z == nz - 1)));
                        if (!wall) h[q] = gb[(kk * 3 + j) * plane + zs3[kk] * ny + ys3[j]];
                    }
            }
            const bool walls = ((bx == BC_NOSLIP || bx == BC_FREESLIP) && (x == 0 || x == nx - 1)) ||
                               ((by == BC_NOSLIP || by == BC_FREESLIP) && (y == 0 || y == ny - 1)) ||
                               ((bz == BC_NOSLIP || bz == BC_FREESLIP) && (z == 0 || z == nz - 1));
            if (walls) {
                float hl[27];
#pragma unroll
                for (int q = 0; q < 27; ++q) hl[q] = h[q];
                boundary_patch<T>(D, src, x, y, z, step, hl);
#pragma unroll
                for (int q = 0; q < 27; ++q) h[q] = hl[q];
            }
            if (bx == BC_INOUT && x == 0) write_inlet_ghost(D, step + 1, y, z);
            float F[3] = {D->body[0], D->body[1], D->body[2]};
            if (rotor_tile) rotor_force(D, step, x, y, z, n_cull, s_pos, s_frc, s_tag, F);
            float m, jx, jy, jz;
            if (COLL == COLL_CUMULANT)
                collide_cumulant(h, F[0], F[1], F[2], D->omega, m, jx, jy, jz);
            else
                collide_srt_smag(h, F[0], F[1], F[2], D->tau0, D->smag_c2, m, jx, jy, jz);
            o_m += m;
            o_jx += jx;
            o_jy += jy;
            o_jz += jz;
            const unsigned cell = ((unsigned)z * (unsigned)ny + (unsigned)y) * (unsigned)nx + (unsigned)x;
#pragma unroll
            for (int q = 0; q < 27; ++q) Io<T>::st(dst + ((unsigned)q * uN + cell), h[q]);
        }
        // diagnostic step: this segment's FP64 sums go to its own lattice
        if (diag) {
            double v[4] = {o_m, o_jx, o_jy, o_jz};
            o_m = o_jx = o_jy = o_jz = 0.0f;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) v[kk] += __shfl_xor_sync(0xFFFFFFFFu, v[kk], o);
            if ((tid & 31) == 0)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) s_red[tid >> 5][kk] = v[kk];
            __syncthreads();
            if (tid == 0)
                for (int kk = 0; kk < 4; ++kk) {
                    double sum = 0.0;
                    for (int w = 0; w < (W >> 5); ++w) sum += s_red[w][kk];
                    atomicAdd(D->diag_acc + kk, sum);
                }
        }
    }
    // after a failed wait: the copies still in flight (segments k .. issued - 1)
    // land before the CTA exits, each wait bounded again, by the full limit
    // whatever the bound of the step's own waits
    if (s_abort) {
        __syncthreads();
        if (tid == 0)
            for (unsigned j = k; j < issued; ++j) (void)mbar_wait(s_full + j % S, (j / S) & 1u, kWaitCycles);
        __syncthreads();
    }
    // diagnostic step: the last CTA closes the sums of every lattice
    if (diag && tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(A.diag_done, 1u);
        if (prev == gridDim.x - 1u) {
            __threadfence();
            for (int i = 0; i < A.n_inst; ++i) {
                const DevDomain* Di = A.dom + i;
                bool finite = true;
                for (int kk = 0; kk < 4; ++kk) {
                    const double sum = __ldcg(Di->diag_acc + kk);
                    Di->diag_res[kk] = sum;
                    Di->diag_acc[kk] = 0.0;
                    if (!isfinite(sum)) finite = false;
                }
                Di->diag_res[4] = (double)step;
                if (!finite) atomicOr(Di->err, ERR_NONFINITE);
            }
            *A.diag_done = 0u;
        }
    }
}

// The actuator line as its own launch: CTA b of a lattice evaluates its
// elements [32 b, 32 b + 32), and the last of the lattice's CTAs to finish adds
// up the per-rotor loads.  In a time step it follows the rotor launch: it lets
// the step's next launch start at once, forms the blade geometry and kernel
// normalisers, then waits on the device until the rotor tiles (which write the
// cells it samples and the box force) are done.  What it reads before that
// wait (the step counter, the turbines' parameters) was written before the
// rotor launch, which starts only after the previous step has completed.
template <typename T>
__global__ void __launch_bounds__(256) k_alm(const AlmArgs A)
{
    asm volatile("griddepcontrol.launch_dependents;");
    __shared__ int s_last;
    int inst = 0;
    while (inst + 1 < A.n_inst && A.cta_off[inst + 1] <= (int)blockIdx.x) ++inst;
    const DevDomain* D = A.dom + inst;
    const int lb = (int)blockIdx.x - A.cta_off[inst];
    const int nb = A.cta_off[inst + 1] - A.cta_off[inst];
    const long long step = A.step_slot ? __ldcg(A.step_slot + A.slot) + 1 : A.step;
    alm_block<T>(D, (const T*)D->f[A.array], step, A.swapped, lb * kAlmBlock);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(D->rotor_counter, 1u);
        s_last = prev == (unsigned)nb - 1u ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        alm_loads(D, step);
        if (tid == 0) *D->rotor_counter = 0u;
    }
}

// Inlet ghost populations of every column for step `step` (after a state change).
__global__ void k_inflow(const DevDomain* D, long long step)
{
    const int plane = D->ny * D->nz;
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < plane; col += gridDim.x * blockDim.x)
        write_inlet_ghost(D, step, col % D->ny, col / D->ny);
}

// f = feq(rho, u) + fneq as offsets, from device copies of the caller's FP64
// rho and u (drho = rho - 1 and u rounded to FP32 here) and FP32 fneq.
// u = nullptr: the mean inflow profile when inflow_mean, else 0.
template <typename T>
__global__ void k_init(const DevDomain* D, const double* rho, const double* u, const float* fneq, int parity,
                       int inflow_mean)
{
    const long long N = D->N;
    T* dst = (T*)D->f[parity];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float ux = 0.f, uy = 0.f, uz = 0.f;
        if (u) {
            ux = (float)u[i];
            uy = (float)u[N + i];
            uz = (float)u[2 * N + i];
        } else if (inflow_mean) {
            const int z = (int)(i / ((long long)D->nx * D->ny));
            double scale = 1.0;
            if (D->inflow_kind == 1) scale = log((z + 0.5) / D->z0) * D->inv_log_zref_z0;
            ux = (float)(D->u_ref[0] * scale);
            uy = (float)(D->u_ref[1] * scale);
            uz = (float)(D->u_ref[2] * scale);
        }
        float E[27];
        feq_offsets(rho ? (float)(rho[i] - 1.0) : 0.0f, ux, uy, uz, E);
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            float v = E[q];
            if (fneq) v += fneq[(size_t)q * N + i];
            Io<T>::st(dst + (size_t)q * N + i, v);
        }
    }
}

// rho = sum f*, u = (sum c f* - F/2)/rho with F the force of the last collision.
template <typename T>
__global__ void k_moments(const DevDomain* D, int parity, double* rho, double* u)
{
    const long long N = D->N;
    const T* f = (const T*)D->f[parity];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float h[27];
#pragma unroll
        for (int q = 0; q < 27; ++q) h[q] = Io<T>::ldcg(f + (size_t)q * N + i);
        const Moments M = raw_moments(h);
        const int x = (int)(i % D->nx);
        const int y = (int)((i / D->nx) % D->ny);
        const int z = (int)(i / ((long long)D->nx * D->ny));
        float F[3] = {D->body[0], D->body[1], D->body[2]};
        alm_box_force(D, x, y, z, F);
        const double r = 1.0 + (double)M.drho;
        rho[i] = r;
        u[i] = ((double)M.jx - 0.5 * (double)F[0]) / r;
        u[N + i] = ((double)M.jy - 0.5 * (double)F[1]) / r;
        u[2 * N + i] = ((double)M.jz - 0.5 * (double)F[2]) / r;
    }
}

// rho and u at listed cells, as k_moments computes them.
template <typename T>
__global__ void k_probe(const DevDomain* D, int parity, const long long* cells, int n, double* out)
{
    const long long N = D->N;
    const T* f = (const T*)D->f[parity];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long long i = cells[k];
        float h[27];
#pragma unroll
        for (int q = 0; q < 27; ++q) h[q] = Io<T>::ldcg(f + (size_t)q * N + i);
        const Moments M = raw_moments(h);
        const int x = (int)(i % D->nx);
        const int y = (int)((i / D->nx) % D->ny);
        const int z = (int)(i / ((long long)D->nx * D->ny));
        float F[3] = {D->body[0], D->body[1], D->body[2]};
        alm_box_force(D, x, y, z, F);
        const double r = 1.0 + (double)M.drho;
        out[4 * k] = r;
        out[4 * k + 1] = ((double)M.jx - 0.5 * (double)F[0]) / r;
        out[4 * k + 2] = ((double)M.jy - 0.5 * (double)F[1]) / r;
        out[4 * k + 3] = ((double)M.jz - 0.5 * (double)F[2]) / r;
    }
}

// One PDF plane as absolute FP64 populations w + h (read-out, checkpoints) and back
// (h = f - w rounded to FP32, then to the storage type).
template <typename T>
__global__ void k_plane_to_f64(const T* src, double* dst, long long n, double w)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = w + (double)Io<T>::ldcg(src + i);
}

template <typename T>
__global__ void k_plane_from_f64(const double* src, T* dst, long long n, double w)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Io<T>::st(dst + i, (float)(src[i] - w));
}

// ------------------------------------------------------------------ launchers

static int grid_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    const long long cap = 152LL * 16;
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

// A launch that may start while the kernel before it on the stream still runs
// (programmatic stream serialization): as soon as every CTA of that kernel has
// signalled griddepcontrol.launch_dependents.
static cudaError_t launch_dependent(void (*kernel)(StepArgs), dim3 grid, dim3 block, cudaStream_t s,
                                    const StepArgs& a)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

// The paired in-place kernel for a collision, storage and step parity
// (16-bit storage); nullptr where it is not built.
static cudaError_t launch_dependent_bulk(void (*kernel)(StepArgs, BulkParams), dim3 grid, dim3 block, cudaStream_t s,
                                         const StepArgs& a, const BulkParams& p);

template <int C, typename T, bool O>
static void (*paired_aa(bool single))(StepArgs, BulkParams)
{
    if constexpr (sizeof(T) == 2) return single ? k_step_aa2<C, T, O, true> : k_step_aa2<C, T, O, false>;
    else return nullptr;
}

cudaError_t launch_step_aa(int coll, int store, dim3 grid, dim3 block, cudaStream_t s, const StepArgs& a, bool odd,
                           bool rotor, bool dependent, const BulkParams* pairs)
{
#define LBM_AA_ONE(C, T, O)                                                                        \
    if (pairs && !rotor) {                                                                         \
        void (*k2)(StepArgs, BulkParams) = paired_aa<C, T, O>(a.n_inst == 1);                      \
        if (!k2) return cudaErrorInvalidValue;                                                     \
        const dim3 b2(block.x / 2, block.y);                                                       \
        if (dependent) return launch_dependent_bulk(k2, grid, b2, s, a, *pairs);                   \
        k2<<<grid, b2, 0, s>>>(a, *pairs);                                                         \
    } else if (rotor) k_step_aa<C, T, O, true><<<grid, block, 0, s>>>(a);                          \
    else if (dependent) return launch_dependent(k_step_aa<C, T, O, false>, grid, block, s, a);     \
    else k_step_aa<C, T, O, false><<<grid, block, 0, s>>>(a);
#define LBM_AA_CASE(C, S, T)                         \
    if (coll == C && store == S) {                   \
        if (odd) { LBM_AA_ONE(C, T, true) }          \
        else { LBM_AA_ONE(C, T, false) }             \
        return cudaGetLastError();                   \
    }
    LBM_AA_CASE(COLL_CUMULANT, STORE_FP32, float)
    LBM_AA_CASE(COLL_CUMULANT, STORE_BF16, __nv_bfloat16)
    LBM_AA_CASE(COLL_CUMULANT, STORE_FP16, __half)
    LBM_AA_CASE(COLL_SRT_SMAG, STORE_FP32, float)
    LBM_AA_CASE(COLL_SRT_SMAG, STORE_BF16, __nv_bfloat16)
    LBM_AA_CASE(COLL_SRT_SMAG, STORE_FP16, __half)
#undef LBM_AA_CASE
#undef LBM_AA_ONE
    return cudaErrorInvalidValue;
}

cudaError_t launch_outlet_fill(int store, const DevDomain* d_dom_inst, const DevDomain& h, long long step, cudaStream_t s)
{
    const int g = grid_for((long long)h.ny * h.nz, 256);
    if (store == STORE_FP32) k_outlet_fill<float><<<g, 256, 0, s>>>(d_dom_inst, step);
    else if (store == STORE_BF16) k_outlet_fill<__nv_bfloat16><<<g, 256, 0, s>>>(d_dom_inst, step);
    else k_outlet_fill<__half><<<g, 256, 0, s>>>(d_dom_inst, step);
    return cudaGetLastError();
}

static cudaError_t launch_dependent_bulk(void (*kernel)(StepArgs, BulkParams), dim3 grid, dim3 block, cudaStream_t s,
                                         const StepArgs& a, const BulkParams& p)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a, p);
}

// The paired bulk kernel for a collision and storage (16-bit storage); false
// where it is not built.
template <int C, typename T>
static bool paired_form(void (*&kb)(StepArgs, BulkParams), bool diag, bool single)
{
    if constexpr (sizeof(T) == 2) {
        kb = diag ? (single ? k_bulk2<C, T, true, true> : k_bulk2<C, T, true, false>)
                  : (single ? k_bulk2<C, T, false, true> : k_bulk2<C, T, false, false>);
        return true;
    } else {
        (void)kb;
        (void)diag;
        (void)single;
        return false;
    }
}

cudaError_t launch_step(int coll, int store, dim3 grid, dim3 block, cudaStream_t s, const StepArgs& a, bool rotor,
                        bool dependent, const BulkParams* bulk, bool diag_step, bool pairs)
{
    const bool march = a.tile_z > 1;
#define LBM_STEP_CASE(C, S, T)                                                                        \
    if (coll == C && store == S) {                                                                    \
        if (a.staged) {                                                                               \
            const size_t smem = bulk_smem_bytes((int)block.x, (int)sizeof(T));                        \
            k_step_staged<C, T><<<grid, block, smem, s>>>(a);                                         \
        } else if (march) {                                                                           \
            if (rotor) k_step<C, T, true, true><<<grid, block, 0, s>>>(a);                            \
            else if (dependent) return launch_dependent(k_step<C, T, true, false>, grid, block, s, a);  \
            else k_step<C, T, true, false><<<grid, block, 0, s>>>(a);                                 \
        } else if (rotor) {                                                                           \
            k_step<C, T, false, true><<<grid, block, 0, s>>>(a);                                      \
        } else if (!bulk) {                                                                           \
            if (dependent) return launch_dependent(k_step<C, T, false, false>, grid, block, s, a);    \
            k_step<C, T, false, false><<<grid, block, 0, s>>>(a);                                     \
        } else {                                                                                      \
            void (*kb)(StepArgs, BulkParams) =                                                        \
                diag_step ? (a.n_inst == 1 ? k_bulk<C, T, true, true> : k_bulk<C, T, true, false>)    \
                          : (a.n_inst == 1 ? k_bulk<C, T, false, true> : k_bulk<C, T, false, false>); \
            dim3 blk = block;                                                                         \
            if (pairs) {                                                                              \
                if (!paired_form<C, T>(kb, diag_step, a.n_inst == 1)) return cudaErrorInvalidValue;  \
                blk.x = block.x / 2;                                                                  \
            }                                                                                         \
            if (dependent) return launch_dependent_bulk(kb, grid, blk, s, a, *bulk);                  \
            kb<<<grid, blk, 0, s>>>(a, *bulk);                                                        \
        }                                                                                             \
        return cudaGetLastError();                                                                    \
    }
    LBM_STEP_CASE(COLL_CUMULANT, STORE_FP32, float)
    LBM_STEP_CASE(COLL_CUMULANT, STORE_BF16, __nv_bfloat16)
    LBM_STEP_CASE(COLL_CUMULANT, STORE_FP16, __half)
    LBM_STEP_CASE(COLL_SRT_SMAG, STORE_FP32, float)
    LBM_STEP_CASE(COLL_SRT_SMAG, STORE_BF16, __nv_bfloat16)
    LBM_STEP_CASE(COLL_SRT_SMAG, STORE_FP16, __half)
#undef LBM_STEP_CASE
    return cudaErrorInvalidValue;
}

// Resident CTAs per SM of the staged kernel for a block width (persistent grid),
// raising its dynamic shared memory limit when needed.
int staged_blocks_per_sm(int coll, int store, int width)
{
    int n = 0;
#define LBM_OCC_CASE(C, S, T)                                                                                    \
    if (coll == C && store == S) {                                                                               \
        const size_t smem = bulk_smem_bytes(width, (int)sizeof(T));                                              \
        if (cudaFuncSetAttribute(k_step_staged<C, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != \
            cudaSuccess)                                                                                         \
            return 0;                                                                                            \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_staged<C, T>, width, smem) != cudaSuccess)  \
            return 0;                                                                                            \
        return n;                                                                                                \
    }
    LBM_OCC_CASE(COLL_CUMULANT, STORE_FP32, float)
    LBM_OCC_CASE(COLL_CUMULANT, STORE_BF16, __nv_bfloat16)
    LBM_OCC_CASE(COLL_CUMULANT, STORE_FP16, __half)
    LBM_OCC_CASE(COLL_SRT_SMAG, STORE_FP32, float)
    LBM_OCC_CASE(COLL_SRT_SMAG, STORE_BF16, __nv_bfloat16)
    LBM_OCC_CASE(COLL_SRT_SMAG, STORE_FP16, __half)
#undef LBM_OCC_CASE
    return n;
}

cudaError_t launch_alm(int store, const AlmArgs& a, cudaStream_t s, bool dependent)
{
    const int grid = a.cta_off[a.n_inst];
    if (grid == 0) return cudaSuccess;
    void (*k)(AlmArgs) = store == STORE_FP32 ? k_alm<float> : (store == STORE_BF16 ? k_alm<__nv_bfloat16> : k_alm<__half>);
    if (!dependent) {
        k<<<grid, 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

cudaError_t launch_inflow(const DevDomain* d_dom_inst, const DevDomain& h, long long step, cudaStream_t s)
{
    k_inflow<<<grid_for((long long)h.ny * h.nz, 256), 256, 0, s>>>(d_dom_inst, step);
    return cudaGetLastError();
}

cudaError_t launch_init(int store, const DevDomain* d_dom_inst, const DevDomain& h, const double* rho, const double* u,
                        const float* fneq, int parity, int inflow_mean, cudaStream_t s)
{
    const int g = grid_for(h.N, 256);
    if (store == STORE_FP32) k_init<float><<<g, 256, 0, s>>>(d_dom_inst, rho, u, fneq, parity, inflow_mean);
    else if (store == STORE_BF16) k_init<__nv_bfloat16><<<g, 256, 0, s>>>(d_dom_inst, rho, u, fneq, parity, inflow_mean);
    else k_init<__half><<<g, 256, 0, s>>>(d_dom_inst, rho, u, fneq, parity, inflow_mean);
    return cudaGetLastError();
}

cudaError_t launch_moments(int store, const DevDomain* d_dom_inst, const DevDomain& h, int parity, double* rho,
                           double* u, cudaStream_t s)
{
    const int g = grid_for(h.N, 256);
    if (store == STORE_FP32) k_moments<float><<<g, 256, 0, s>>>(d_dom_inst, parity, rho, u);
    else if (store == STORE_BF16) k_moments<__nv_bfloat16><<<g, 256, 0, s>>>(d_dom_inst, parity, rho, u);
    else k_moments<__half><<<g, 256, 0, s>>>(d_dom_inst, parity, rho, u);
    return cudaGetLastError();
}

cudaError_t launch_probe(int store, const DevDomain* d_dom_inst, int parity, const long long* cells, int n, double* out,
                         cudaStream_t s)
{
    const int g = grid_for(n, 128);
    if (store == STORE_FP32) k_probe<float><<<g, 128, 0, s>>>(d_dom_inst, parity, cells, n, out);
    else if (store == STORE_BF16) k_probe<__nv_bfloat16><<<g, 128, 0, s>>>(d_dom_inst, parity, cells, n, out);
    else k_probe<__half><<<g, 128, 0, s>>>(d_dom_inst, parity, cells, n, out);
    return cudaGetLastError();
}

cudaError_t launch_plane_to_f64(int store, const void* src, double* dst, long long n, double w, cudaStream_t s)
{
    const int g = grid_for(n, 256);
    if (store == STORE_FP32) k_plane_to_f64<float><<<g, 256, 0, s>>>((const float*)src, dst, n, w);
    else if (store == STORE_BF16) k_plane_to_f64<__nv_bfloat16><<<g, 256, 0, s>>>((const __nv_bfloat16*)src, dst, n, w);
    else k_plane_to_f64<__half><<<g, 256, 0, s>>>((const __half*)src, dst, n, w);
    return cudaGetLastError();
}

cudaError_t launch_plane_from_f64(int store, const double* src, void* dst, long long n, double w, cudaStream_t s)
{
    const int g = grid_for(n, 256);
    if (store == STORE_FP32) k_plane_from_f64<float><<<g, 256, 0, s>>>(src, (float*)dst, n, w);
    else if (store == STORE_BF16) k_plane_from_f64<__nv_bfloat16><<<g, 256, 0, s>>>(src, (__nv_bfloat16*)dst, n, w);
    else k_plane_from_f64<__half><<<g, 256, 0, s>>>(src, (__half*)dst, n, w);
    return cudaGetLastError();
}

}  // namespace lbmgb
