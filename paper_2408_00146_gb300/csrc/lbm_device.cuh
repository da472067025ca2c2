// lbm_device.cuh -- device-side helpers shared by the step kernels of
// lbm_kernels.cu (tile kernels, observation, initial state) and lbm_stream.cu
// (y-streaming kernels): lattice constants, the surface tension law, the
// isotropic gradient, the factorised central-moment transform, 16-bit
// conversions and the TMA / mbarrier primitives with their bounded wait.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "lbm_internal.h"

namespace {

constexpr float kCs2 = 1.0f / 3.0f;
constexpr float kW1 = 1.0f / 9.0f, kW2 = 1.0f / 36.0f;  // D2Q9 weights of axis and diagonal links
// n = grad phi / max(|grad phi|, eps): the normal of Sec. 3 is undefined where
// grad phi vanishes (bubble interiors, whose centre has no gradient direction);
// the floor keeps the sharpening flux M theta n there proportional to grad phi
// instead of following rounding noise.  It acts only where phi (1 - phi) <
// W eps / 4 on the equilibrium profile (the far tails of the interface).
constexpr float kNormalEps = 1e-4f;

__device__ __forceinline__ int wrap(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Source row of a stencil value at physical row y, and which wall image it is
// (-1 bottom, +1 top, 0 none): with walls, rows at and beyond a wall mirror
// about the wall plane (y = 1/2, y = ny - 3/2); without walls y wraps.
__device__ __forceinline__ int src_row(const LbmDev& d, int y, int& side)
{
    side = 0;
    if (!d.walls) return wrap(y, d.ny);
    if (y < 1) {
        side = -1;
        y = 1 - y;
    } else if (y > d.ny - 2) {
        side = 1;
        y = 2 * d.ny - 3 - y;
    }
    // positions farther than one reflection only feed inactive tile slots
    return min(max(y, 1), d.ny - 2);
}

// Stencil ghost of psi at a wall mirror (side -1 below the y=0 wall, +1
// above the y=ny-1 wall): even about the wall plane for zero-flux walls, odd
// about psi_w when psi is held at psi_L / psi_R (psi_bc 1), as T about T_w.
__device__ __forceinline__ float psi_ghost(const LbmDev& d, float psi, int side)
{
    if (d.psi_bc != 1 || side == 0) return psi;
    return 2.0f * (side < 0 ? d.psi_L : d.psi_R) - psi;
}

// The properties rho, mu, alpha are interpolated linearly in phi (Eq. (17))
// with phi clamped to [0, 1] (__saturatef): the conservative phase field
// overshoots 1 by ~1e-3 inside a bubble, which at a density ratio of 1000
// would make rho_B + (phi - 1)(rho_B - rho_A) negative.

// Surface tension law, Eq. (6); ln(1 - psi) with psi clamped to [0, 1-1e-6].
__device__ __forceinline__ float sigma_eos(const LbmDev& d, float T, float psi)
{
    float pc = fminf(fmaxf(psi, 0.0f), 1.0f - 1e-6f);
    float dT = T - d.T_ref;
    return d.sigma0 + d.s0beta_over_Tref * T * log1pf(-pc) + d.sigma_T * dT +
           d.sigma_TT * dT * dT;
}

// Isotropic gradient 3 sum_a w_a e_a X(x + e_a) on a shared-memory array
// (row index = y).
template <int P>
__device__ __forceinline__ void grad_smem(const float (*a)[P], int r, int c, float& gx, float& gy)
{
    const float e = a[r][c + 1], w = a[r][c - 1], n = a[r + 1][c], s = a[r - 1][c];
    const float ne = a[r + 1][c + 1], nw = a[r + 1][c - 1], se = a[r - 1][c + 1],
                sw = a[r - 1][c - 1];
    gx = (1.0f / 3.0f) * (e - w) + (1.0f / 12.0f) * ((ne - nw) + (se - sw));
    gy = (1.0f / 3.0f) * (n - s) + (1.0f / 12.0f) * ((ne - se) + (nw - sw));
}

// Inverse of the factorised central-moment transform: central moments
// c_mn (m along x, n along y) about (ux, uy) to the nine populations.
__device__ __forceinline__ void central_to_pop(float c00, float c10, float c01, float c20,
                                               float c02, float c11, float c21, float c12,
                                               float c22, float ux, float uy, float out[9])
{
    const float uy2 = uy * uy, ux2 = ux * ux;
    // along y: (c_m0, c_m1, c_m2) -> partial x-moments k_m at e_y = -1, 0, +1
    float k0m, k00, k0p, k1m, k10, k1p, k2m, k20, k2p;
#define YPASS(a0, a1, a2, km, kz, kp)                                       \
    kz = (a0) * (1.0f - uy2) - 2.0f * uy * (a1) - (a2);                     \
    kp = 0.5f * ((a0) * (uy2 + uy) + (a1) * (2.0f * uy + 1.0f) + (a2));     \
    km = 0.5f * ((a0) * (uy2 - uy) + (a1) * (2.0f * uy - 1.0f) + (a2));
    YPASS(c00, c01, c02, k0m, k00, k0p)
    YPASS(c10, c11, c12, k1m, k10, k1p)
    YPASS(c20, c21, c22, k2m, k20, k2p)
#undef YPASS
    // along x at each e_y: (k_0, k_1, k_2) -> populations at e_x = -1, 0, +1
#define XPASS(a0, a1, a2, fm, fz, fp)                                       \
    fz = (a0) * (1.0f - ux2) - 2.0f * ux * (a1) - (a2);                     \
    fp = 0.5f * ((a0) * (ux2 + ux) + (a1) * (2.0f * ux + 1.0f) + (a2));     \
    fm = 0.5f * ((a0) * (ux2 - ux) + (a1) * (2.0f * ux - 1.0f) + (a2));
    XPASS(k00, k10, k20, out[3], out[0], out[1])   // e_y = 0
    XPASS(k0p, k1p, k2p, out[6], out[2], out[5])   // e_y = +1
    XPASS(k0m, k1m, k2m, out[7], out[4], out[8])   // e_y = -1
#undef XPASS
}

// Packed FP32 pairs: one FFMA2 / FADD2 / FMUL2 instruction does the
// operation on both lanes, each lane rounded exactly as the scalar operation.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ float sum9(const float v[9])
{
    return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
}
__device__ __forceinline__ float mx9(const float v[9])
{
    return (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
}
__device__ __forceinline__ float my9(const float v[9])
{
    return (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
}


// ---- TMA / mbarrier helpers (sm_90+ PTX) -------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: gives up once limit_ns of wall time have passed (checked
// every 256 polls of the barrier), or after kMaxWaitPolls polls whatever the
// timer says, instead of spinning forever.  A copy that never completes thus
// costs its block about a second and an error flag, not a hung GPU.
constexpr int kMaxWaitPolls = 1 << 24;
constexpr uint64_t kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int i = 1; i < kMaxWaitPolls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 0 && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// One TMA copy of the box {kTileX, kTileY, 36} at (x, y, plane 0) of the
// population tensor [36][ny][nx] into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_tile(uint32_t dst, const CUtensorMap* map, int x, int y,
                                              uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(0), "r"(bar)
        : "memory");
}


template <typename S> __device__ __forceinline__ float s2f(S v);
template <> __device__ __forceinline__ float s2f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float s2f<__nv_bfloat16>(__nv_bfloat16 v)
{
    return __bfloat162float(v);
}
template <typename S> __device__ __forceinline__ S f2s(float v);
template <> __device__ __forceinline__ __half f2s<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 f2s<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}
// Two values of a set pair in one 32-bit word (the first in the low half),
// each rounded to nearest even as f2s rounds it, and back.
template <typename S> __device__ __forceinline__ uint32_t f2s2(float a, float b);
template <> __device__ __forceinline__ uint32_t f2s2<__half>(float a, float b)
{
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}
template <> __device__ __forceinline__ uint32_t f2s2<__nv_bfloat16>(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}
template <typename S> __device__ __forceinline__ float2 s2f2(uint32_t v);
template <> __device__ __forceinline__ float2 s2f2<__half>(uint32_t v)
{
    return __half22float2(*reinterpret_cast<const __half2*>(&v));
}
template <> __device__ __forceinline__ float2 s2f2<__nv_bfloat16>(uint32_t v)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v));
}

// 16-bit storage layout: the sets are stored in pairs, (f, g) and (h, q),
// the pair's two values of a population side by side in one 32-bit word,
// [2 pairs][9 directions][ny][nx][2].  Element of population a of set s at
// node o (N = nx ny nodes).
__device__ __forceinline__ size_t dev_index(int s, int a, size_t N, size_t o)
{
    return (((size_t)(s >> 1) * 9 + a) * N + o) * 2 + (s & 1);
}

__device__ __forceinline__ constexpr float w_of_dir(int a)
{
    return a == 0 ? 4.0f / 9.0f : (a <= 4 ? kW1 : kW2);
}
// Integer weights of 16-bit storage: population a = k_a m + deviation with
// m = M/36 per node, k_a = 36 w_a (16, 4, 1) exact in FP32, so that the nine
// weights sum to 36 exactly and a node's populations sum to 36 m + sum dev.
__device__ __forceinline__ constexpr float k_of_dir(int a)
{
    return a == 0 ? 16.0f : (a <= 4 ? 4.0f : 1.0f);
}
constexpr float kInv36 = 1.0f / 36.0f;
__device__ __forceinline__ constexpr int ex_dir(int a)
{
    return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__device__ __forceinline__ constexpr int ey_dir(int a)
{
    return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}


}  // namespace
