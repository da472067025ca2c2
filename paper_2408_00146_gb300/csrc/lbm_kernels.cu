// lbm_kernels.cu -- sm_103a kernels of the fused collide-and-stream step of
// the coupled central-moment lattice Boltzmann system of arXiv 2408.00146.
//
// Data layout in HBM (structure of arrays, x fastest):
//   populations  pop[set][alpha][y][x], set 0 = f (phase field, App. B),
//                1 = g (pressure/velocity, App. C), 2 = h (energy, App. D),
//                3 = q (surfactant, App. E); FP32; two buffers (ping-pong);
//   fields       fld[k][y][x], k = phi, u_x, u_y, p, T, psi; FP32.
// A buffer holds the post-streaming populations of one time level.  One step
// reads them at the node (coalesced), computes the macroscopic fields of the
// tile plus a two-node halo in shared memory, evaluates the isotropic
// stencils, forces and the four central-moment collisions in registers, and
// pushes the post-collision populations to the neighbours of the other
// buffer (halfway bounce-back / anti-bounce-back at the walls).
//
// The moment transforms use the factorised form of the binomial frame change
// of Eq. (24b)/(46): central moments are taken first along x, then along y,
// and the inverse runs the same one-dimensional maps backwards.  Each
// collision is applied as an increment: the change of the central moments is
// mapped back to the populations and added to them, which keeps the conserved
// zeroth moments to one rounding per population instead of re-synthesising the
// populations from a rounded sum.
#include "lbm_internal.h"
#include "lbm_device.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

namespace {


// Equilibrium-type scalar scheme (f, h, q): post-collision central moments
// (s, a, b, s/3, s/3, 0, 0, 0, s/9).
__device__ __forceinline__ void scalar_post(float s, float a, float b, float ux, float uy,
                                            float out[9])
{
    central_to_pop(s, a, b, kCs2 * s, kCs2 * s, 0.0f, 0.0f, 0.0f, kCs2 * kCs2 * s, ux, uy,
                   out);
}

// Forward factorised transform: populations to the nine central moments about
// (ux, uy), first along x at each e_y, then along y; c[] in the order
// 00, 10, 01, 20, 02, 11, 21, 12, 22.
__device__ __forceinline__ void pop_to_central(const float f[9], float ux, float uy, float c[9])
{
    float k0[3], k1[3], k2[3];  // index 0: e_y = -1, 1: e_y = 0, 2: e_y = +1
#define XFWD(fm, fz, fp, j)                                   \
    {                                                         \
        const float d = (fp) - (fm), s = (fp) + (fm);         \
        k0[j] = s + (fz);                                     \
        k1[j] = d - ux * k0[j];                               \
        k2[j] = s - ux * (d + k1[j]);                         \
    }
    XFWD(f[7], f[4], f[8], 0)
    XFWD(f[3], f[0], f[1], 1)
    XFWD(f[6], f[2], f[5], 2)
#undef XFWD
#define YFWD(k, c0, c1, c2)                                   \
    {                                                         \
        const float d = k[2] - k[0], s = k[2] + k[0];         \
        c0 = s + k[1];                                        \
        c1 = d - uy * c0;                                     \
        c2 = s - uy * (d + c1);                               \
    }
    YFWD(k0, c[0], c[2], c[4])
    YFWD(k1, c[1], c[5], c[7])
    YFWD(k2, c[3], c[6], c[8])
#undef YFWD
}

// Adds to the populations the change of their central moments: f += P^-1
// F(-u) dc, i.e. the collision applied as an increment, so that the zeroth
// moment is carried by the stored populations rather than re-synthesised from
// its rounded sum.
__device__ __forceinline__ void add_central_increment(float f[9], const float dc[9], float ux,
                                                      float uy)
{
    float df[9];
    central_to_pop(dc[0], dc[1], dc[2], dc[3], dc[4], dc[5], dc[6], dc[7], dc[8], ux, uy, df);
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a] += df[a];
}

// Collision of a scalar scheme (App. B, D, E): zeroth moment kept, first-order
// central moments relaxed with rate w towards (e10, e01), every higher moment
// set to its equilibrium (s/3, s/3, 0, 0, 0, s/9).
__device__ __forceinline__ void scalar_collide(float f[9], float s, float e10, float e01, float w,
                                               float ux, float uy)
{
    float c[9];
    pop_to_central(f, ux, uy, c);
    float dc[9];
    dc[0] = 0.0f;
    dc[1] = w * (e10 - c[1]);
    dc[2] = w * (e01 - c[2]);
    dc[3] = kCs2 * s - c[3];
    dc[4] = kCs2 * s - c[4];
    dc[5] = -c[5];
    dc[6] = -c[6];
    dc[7] = -c[7];
    dc[8] = kCs2 * kCs2 * s - c[8];
    add_central_increment(f, dc, ux, uy);
}

enum Mode { kStep = 0, kFields = 1 };

// Neighbour offsets (within one population plane) of node idx = y*nx + x,
// x wrapping periodically and y wrapping without walls.
struct Nbr {
    int o[9];
};

__device__ __forceinline__ Nbr neighbours(const LbmDev& d, int x, int y)
{
    const int xw = (x == 0) ? d.nx - 1 : x - 1;
    const int xe = (x + 1 == d.nx) ? 0 : x + 1;
    const int r = y * d.nx;
    int rs = r - d.nx, rn = r + d.nx;
    if (!d.walls) {
        if (y == 0) rs = (d.ny - 1) * d.nx;
        if (y == d.ny - 1) rn = 0;
    }
    Nbr n;
    n.o[0] = r + x;
    n.o[1] = r + xe;
    n.o[2] = rn + x;
    n.o[3] = r + xw;
    n.o[4] = rs + x;
    n.o[5] = rn + xe;
    n.o[6] = rn + xw;
    n.o[7] = rs + xw;
    n.o[8] = rs + xe;
    return n;
}

// Push the nine post-collision populations of one set to the neighbours in
// dst_set (plane stride N).  wall = -1 (bottom fluid row), +1 (top fluid row)
// or 0; a population headed into a wall row returns to the node in the
// opposite direction (halfway bounce-back, or anti-bounce-back with the wall
// temperature Tw for the energy set).  wall is uniform across a warp.
template <bool kEnergy>
__device__ __forceinline__ void store_set(float* __restrict__ dst_set, int N, const Nbr& nb,
                                          const float v[9], int wall, float Tw)
{
    const int o0 = nb.o[0];
    dst_set[o0] = v[0];
    dst_set[N + nb.o[1]] = v[1];
    dst_set[3 * N + nb.o[3]] = v[3];
    if (wall == 0) {
        dst_set[2 * N + nb.o[2]] = v[2];
        dst_set[4 * N + nb.o[4]] = v[4];
        dst_set[5 * N + nb.o[5]] = v[5];
        dst_set[6 * N + nb.o[6]] = v[6];
        dst_set[7 * N + nb.o[7]] = v[7];
        dst_set[8 * N + nb.o[8]] = v[8];
    } else if (wall < 0) {  // e_y = -1 hits the bottom wall: 4 -> 2, 7 -> 5, 8 -> 6
        dst_set[2 * N + nb.o[2]] = v[2];
        dst_set[5 * N + nb.o[5]] = v[5];
        dst_set[6 * N + nb.o[6]] = v[6];
        dst_set[2 * N + o0] = kEnergy ? -v[4] + 2.0f * kW1 * Tw : v[4];
        dst_set[5 * N + o0] = kEnergy ? -v[7] + 2.0f * kW2 * Tw : v[7];
        dst_set[6 * N + o0] = kEnergy ? -v[8] + 2.0f * kW2 * Tw : v[8];
    } else {                // e_y = +1 hits the top wall: 2 -> 4, 5 -> 7, 6 -> 8
        dst_set[4 * N + nb.o[4]] = v[4];
        dst_set[7 * N + nb.o[7]] = v[7];
        dst_set[8 * N + nb.o[8]] = v[8];
        dst_set[4 * N + o0] = kEnergy ? -v[2] + 2.0f * kW1 * Tw : v[2];
        dst_set[7 * N + o0] = kEnergy ? -v[5] + 2.0f * kW2 * Tw : v[5];
        dst_set[8 * N + o0] = kEnergy ? -v[6] + 2.0f * kW2 * Tw : v[6];
    }
}

// Wrapped column of x for lattices at least as wide as a tile plus its halo;
// narrower lattices take the modulo.
__device__ __forceinline__ int wrap_x(const LbmDev& d, int x)
{
    if (d.nx >= kTileX + 4) return x < 0 ? x + d.nx : (x >= d.nx ? x - d.nx : x);
    return wrap(x, d.nx);
}

// ---- per-tile pieces shared by the step kernels -------------------------------------

// The 36 staged populations of one node: p[a * stride], a = 9 set + alpha.
struct OwnPops {
    const float* p;
    int stride;
    __device__ __forceinline__ float operator()(int a) const { return p[a * stride]; }
};

// Shared-memory views of one tile: its own populations [36][TY][TX] and the
// macroscopic fields on the tile plus halo (phi with two nodes of halo, the
// rest with one).
struct TileSmem {
    float (*pop)[kTileY][kTileX];
    float (*phi)[kTileX + 4];
    float (*sig)[kTileX + 2];
    float (*phs)[kTileX + 2];
    float (*nrmx)[kTileX + 2];
    float (*nrmy)[kTileX + 2];
};

struct NodeMoments {
    float phi, T, psi, pst, jx, jy;
};

// Moments of the own node (Eqs. (28), (34), (39), (44)) from the staged
// populations; phi, sigma(T, psi) and p* - rho c_s^2 go to the field tiles.
// side != 0: the slot holds a wall mirror, whose temperature is 2 T_w - T.
__device__ __forceinline__ NodeMoments own_moments(const LbmDev& d, const TileSmem& sm,
                                                   const OwnPops& own, int tx, int ty, int side)
{
    NodeMoments m;
    float v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = own(a);
    m.phi = sum9(v);
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = own(9 + a);
    m.pst = sum9(v);
    m.jx = mx9(v);
    m.jy = my9(v);
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = own(18 + a);
    m.T = sum9(v);
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = own(27 + a);
    m.psi = sum9(v);
    float Tg = m.T;
    if (side < 0) Tg = 2.0f * d.T_H - m.T;
    if (side > 0) Tg = 2.0f * d.T_C - m.T;
    sm.phi[ty + 2][tx + 2] = m.phi;
    sm.sig[ty + 1][tx + 1] = sigma_eos(d, Tg, psi_ghost(d, m.psi, side));
    sm.phs[ty + 1][tx + 1] = m.pst - (d.rhoA + __saturatef(m.phi) * d.drho) * kCs2;
    return m;
}

// Field values of one halo slot (ex, ey) from its sums: phi always; sigma
// and p* - rho c_s^2 for the inner ring.
__device__ __forceinline__ void halo_fields(const LbmDev& d, const TileSmem& sm, int ex, int ey,
                                            bool ring1, int side, float ph, float ps, float Th,
                                            float sp)
{
    sm.phi[ey][ex] = ph;
    if (ring1) {
        if (side < 0) Th = 2.0f * d.T_H - Th;
        if (side > 0) Th = 2.0f * d.T_C - Th;
        sm.sig[ey - 1][ex - 1] = sigma_eos(d, Th, psi_ghost(d, sp, side));
        sm.phs[ey - 1][ex - 1] = ps - (d.rhoA + __saturatef(ph) * d.drho) * kCs2;
    }
}

// Unit normals n = grad phi / max(|grad phi|, eps) on the tile + 1-node halo.
__device__ __forceinline__ void normals_pass(const TileSmem& sm, int tid, int nthreads)
{
    constexpr int RW = kTileX + 2, RH = kTileY + 2;
    for (int i = tid; i < RW * RH; i += nthreads) {
        const int cx = i % RW, cy = i / RW;
        float gxp, gyp;
        grad_smem<kTileX + 4>(sm.phi, cy + 1, cx + 1, gxp, gyp);
        const float inv = fminf(rsqrtf(gxp * gxp + gyp * gyp), 1.0f / kNormalEps);
        sm.nrmx[cy][cx] = gxp * inv;
        sm.nrmy[cy][cx] = gyp * inv;
    }
}

// Where node_update puts the post-collision populations of set `set`
// (0 f, 1 g, 2 h, 3 q; M = its zeroth moment after the collision): FP32
// populations pushed to the neighbours.  put returns the rest-state moment the
// stored values refer to (unused here); finish receives the four of a node.
struct StoreF32 {
    float* dst;
    template <bool kEnergy>
    __device__ __forceinline__ float put(int set, int N, const Nbr& nb, const float v[9], float M,
                                         int wall, float Tw) const
    {
        store_set<kEnergy>(dst + (size_t)set * 9 * N, N, nb, v, wall, Tw);
        return M;
    }
    __device__ __forceinline__ void finish(int, float, float, float, float) const {}
};

// Stencils, forces, velocity and pressure (Sec. 3, App. C), then the four
// collisions and the push to the neighbours (or, in kFields mode, the fields).
template <int kMode, class Store, class Own>
__device__ __forceinline__ void node_update(const LbmDev& d, const TileSmem& sm,
                                            const NodeMoments& m, const Own& own,
                                            const Store& st, float* __restrict__ fdst, int tx,
                                            int ty, int gx, int gy)
{
    const int N = d.nx * d.ny;
    const int r = ty + 1, c = tx + 1;
    float gpx, gpy;
    grad_smem<kTileX + 4>(sm.phi, ty + 2, tx + 2, gpx, gpy);
    const float g2 = gpx * gpx + gpy * gpy;
    const float n_x = sm.nrmx[r][c], n_y = sm.nrmy[r][c];
    float dnx_dx, dnx_dy, dny_dx, dny_dy;
    grad_smem<kTileX + 2>(sm.nrmx, r, c, dnx_dx, dnx_dy);
    grad_smem<kTileX + 2>(sm.nrmy, r, c, dny_dx, dny_dy);
    const float kappa = dnx_dx + dny_dy;
    float sgx, sgy, phx, phy;
    grad_smem<kTileX + 2>(sm.sig, r, c, sgx, sgy);
    grad_smem<kTileX + 2>(sm.phs, r, c, phx, phy);
    const float sig = sm.sig[r][c];
    const float ndots = n_x * sgx + n_y * sgy;
    const float deltas = d.deltas_coef * g2;
    const float phi = m.phi, T = m.T, psi = m.psi;
    const float rho = d.rhoA + __saturatef(phi) * d.drho;
    const float inv_rho = __fdividef(1.0f, rho);
    const float Ftx = deltas * (-sig * kappa * n_x + sgx - n_x * ndots) + d.Fext_x;
    const float Fty = deltas * (-sig * kappa * n_y + sgy - n_y * ndots) + d.Fext_y -
                      (rho - d.rhoA) * d.gravity;
    const float Fpx = -phx, Fpy = -phy;
    const float ux = (3.0f * m.jx + 0.5f * Ftx) * inv_rho;
    const float uy = (3.0f * m.jy + 0.5f * Fty) * inv_rho;
    const float Gam = Fpx * ux + Fpy * uy;
    const float p = m.pst + 0.5f * Gam;

    if (kMode == kFields) {
        const int o = gy * d.nx + gx;
        fdst[o] = phi;
        fdst[N + o] = ux;
        fdst[2 * N + o] = uy;
        fdst[3 * N + o] = p;
        fdst[4 * N + o] = T;
        fdst[5 * N + o] = psi;
        return;
    }

    const Nbr nb = neighbours(d, gx, gy);
    const int wall = !d.walls ? 0 : (gy == 1 ? -1 : (gy == d.ny - 2 ? 1 : 0));
    float v[9];
    float Mf, Mg, Mh, Mq;  // rest-state moments the stored populations refer to
    // ---- f: conservative Allen-Cahn (App. B) ---------------------------------------
    {
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = own(a);
        const float theta_m = d.mphi_4_over_W * phi * (1.0f - phi);   // M_phi theta
        scalar_collide(v, phi, theta_m * n_x, theta_m * n_y, d.omega_phi, ux, uy);
        Mf = st.template put<false>(0, N, nb, v, phi, wall, 0.0f);
    }
    // ---- h: energy (App. D), rate from the local thermal diffusivity -----------------
    {
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = own(18 + a);
        const float alpha = d.alphaA + __saturatef(phi) * d.dalpha;
        const float wT = __fdividef(1.0f, 3.0f * alpha + 0.5f);
        scalar_collide(v, T, 0.0f, 0.0f, wT, ux, uy);
        Mh = st.template put<true>(2, N, nb, v, T, wall, wall < 0 ? d.T_H : d.T_C);
    }
    // ---- q: surfactant (App. E) -------------------------------------------------
    {
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = own(27 + a);
        const float dG = (phi - 0.5f) * (d.g_s32 * phi * (1.0f - phi) + d.g_w);
        const float flux = -d.m_psi * psi * (1.0f - psi) * dG;   // times grad phi
        scalar_collide(v, psi, flux * gpx, flux * gpy, d.omega_psi, ux, uy);
        // walls: halfway bounce-back, or anti-bounce-back with psi_L / psi_R
        Mq = d.psi_bc == 1
                 ? st.template put<true>(3, N, nb, v, psi, wall, wall < 0 ? d.psi_L : d.psi_R)
                 : st.template put<false>(3, N, nb, v, psi, wall, 0.0f);
    }
    // ---- g: two-fluid pressure/velocity (App. C) ----------------------------------------
    {
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = own(9 + a);
        const float mu = d.muA + __saturatef(phi) * d.dmu;
        const float wn = __fdividef(1.0f, 3.0f * mu * inv_rho + 0.5f);
        const float vp = p - rho * kCs2;                      // varphi = p - rho c_s^2
        const float ux2 = ux * ux, uy2 = uy * uy;
        float cm[9];
        pop_to_central(v, ux, uy, cm);
        // equilibria (Eq. (31)) and sources (Eq. (32))
        const float e20 = p * kCs2 + vp * ux2, e02 = p * kCs2 + vp * uy2;
        const float e11 = vp * ux * uy;
        const float e21 = -vp * (ux2 + kCs2) * uy;
        const float e12 = -vp * (uy2 + kCs2) * ux;
        // c_s^6 rho + varphi (u_x^2 + c_s^2)(u_y^2 + c_s^2) with the two O(rho)
        // terms cancelled exactly: p c_s^4 + varphi (c_s^2 (u_x^2 + u_y^2) + u_x^2 u_y^2)
        const float e22 = kCs2 * kCs2 * p + vp * (kCs2 * (ux2 + uy2) + ux2 * uy2);
        const float s10 = kCs2 * Ftx - ux * Gam, s01 = kCs2 * Fty - uy * Gam;
        const float s20 = 2.0f * kCs2 * Fpx * ux + (ux2 + kCs2) * Gam;
        const float s02 = 2.0f * kCs2 * Fpy * uy + (uy2 + kCs2) * Gam;
        const float s11 = kCs2 * (Fpx * uy + Fpy * ux) + ux * uy * Gam;
        // relaxation (Eq. (33)) as an increment of the central moments: rate 1
        // for 00, 10, 01, 2s, 21, 12, 22 (new value = equilibrium + source/2),
        // omega_nu for 2d and 11.  With rate 1 the zeroth and first moments
        // change by exactly their source: the equilibrium p + Gam/2 and
        // -varphi u + s/2 differ from the pre-collision p* and j - u p* by
        // Gam/2 and s/2, by the definitions of p and u (Eq. (34)).
        float dc[9];
        dc[0] = Gam;
        dc[1] = s10;
        dc[2] = s01;
        const float d2s = (e20 + e02) + 0.5f * (s20 + s02) - (cm[3] + cm[4]);
        const float k2d = cm[3] - cm[4];
        const float d2d = wn * ((e20 - e02) - k2d) + (1.0f - 0.5f * wn) * (s20 - s02);
        dc[3] = 0.5f * (d2s + d2d);
        dc[4] = 0.5f * (d2s - d2d);
        dc[5] = wn * (e11 - cm[5]) + (1.0f - 0.5f * wn) * s11;
        dc[6] = e21 - cm[6];
        dc[7] = e12 - cm[7];
        dc[8] = e22 - cm[8];
        add_central_increment(v, dc, ux, uy);
        // zeroth moment after the collision: p* + Gamma (dc[0])
        Mg = st.template put<false>(1, N, nb, v, m.pst + Gam, wall, 0.0f);
    }
    st.finish(gy * d.nx + gx, Mf, Mg, Mh, Mq);
}

// ---- one tile per block ---------------------------------------------------------------

// The fused step for the tile (bx, by).  Block = kTileX x kTileY threads, one
// output node each.  The tile's own populations are staged in shared memory:
// by one TMA copy for tiles that lie wholly inside the lattice (kTma: tmap is
// the tensor map of src), else by per-thread loads that also resolve periodic
// images and wall mirrors for the slots past the lattice edge.  Halo sums
// are loaded while the copy is in flight.
template <int kMode, bool kTma>
__device__ __forceinline__ void step_tile(const LbmDev& d, const float* __restrict__ src,
                                          float* __restrict__ dst, const CUtensorMap* tmap,
                                          int* __restrict__ err, int bx, int by)
{
    constexpr int TX = kTileX, TY = kTileY;
    constexpr int EW = TX + 4, EH = TY + 4;
    constexpr int RW = TX + 2, RH = TY + 2;
    __shared__ __align__(128) float s_pop[36][TY][TX];
    __shared__ float s_phi[EH][EW];
    __shared__ float s_sig[RH][RW];
    __shared__ float s_phs[RH][RW];
    __shared__ float s_nx[RH][RW];
    __shared__ float s_ny[RH][RW];
    __shared__ __align__(8) uint64_t s_bar;
    const TileSmem sm{s_pop, s_phi, s_sig, s_phs, s_nx, s_ny};

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int x0 = bx * TX;
    const int fy0 = by * TY;                  // tile origin in fluid-row numbering
    const int N = d.nx * d.ny;
    const int gx = x0 + tx;
    const int gfy = fy0 + ty;
    const bool active = (gx < d.nx) && (gfy < d.nfy);
    const int gy = d.y0 + gfy;
    const bool use_tma = kTma && tmap != nullptr && (x0 + TX <= d.nx) && (fy0 + TY <= d.nfy);
    const uint32_t bar = smem_addr(&s_bar);

    int own_side = 0;
    if (use_tma) {
        if (tid == 0) mbar_init(bar, 1);
        __syncthreads();
        if (tid == 0) {
            mbar_expect_tx(bar, 36u * TX * TY * sizeof(float));
            tma_load_tile(smem_addr(&s_pop[0][0][0]), tmap, x0, d.y0 + fy0, bar);
        }
    } else {
        const int sx = wrap_x(d, gx);
        const int sy = src_row(d, gy, own_side);
        const float* p = src + (sy * d.nx + sx);
#pragma unroll
        for (int a = 0; a < 36; ++a) s_pop[a][ty][tx] = __ldg(p + a * N);
    }

    for (int i = tid; i < EW * EH; i += TX * TY) {
        const int ex = i % EW, ey = i / EW;
        if (ex >= 2 && ex < TX + 2 && ey >= 2 && ey < TY + 2) continue;
        const bool ring1 = ex >= 1 && ex <= TX + 2 && ey >= 1 && ey <= TY + 2;
        int side;
        const int sx = wrap_x(d, x0 + ex - 2);
        const int sy = src_row(d, d.y0 + fy0 + ey - 2, side);
        const float* p = src + (sy * d.nx + sx);
        float v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = __ldg(p + a * N);
        const float ph = sum9(v);
        float ps = 0.0f, Th = 0.0f, sp = 0.0f;
        if (ring1) {
#pragma unroll
            for (int a = 0; a < 9; ++a) v[a] = __ldg(p + (9 + a) * N);
            ps = sum9(v);
#pragma unroll
            for (int a = 0; a < 9; ++a) v[a] = __ldg(p + (18 + a) * N);
            Th = sum9(v);
#pragma unroll
            for (int a = 0; a < 9; ++a) v[a] = __ldg(p + (27 + a) * N);
            sp = sum9(v);
        }
        halo_fields(d, sm, ex, ey, ring1, side, ph, ps, Th, sp);
    }

    if (use_tma) {
        const bool ok = mbar_wait_bounded(bar, 0);
        if (__syncthreads_or(!ok)) {
            // the copy did not complete in time: report it, and keep the block
            // resident for one more bounded wait so that no transfer into its
            // shared memory can outlive it
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait_bounded(bar, 0);
            }
            return;
        }
    }
    const OwnPops own{&s_pop[0][ty][tx], TX * TY};
    const NodeMoments m = own_moments(d, sm, own, tx, ty, own_side);
    __syncthreads();
    normals_pass(sm, tid, TX * TY);
    __syncthreads();
    if (!active) return;
    node_update<kMode>(d, sm, m, own, StoreF32{dst}, dst, tx, ty, gx, gy);
}

template <int kMode, bool kTma>
__global__ void __launch_bounds__(kTileX * kTileY, 4)
    step_kernel(LbmDev d, const float* __restrict__ src, float* __restrict__ dst,
                const __grid_constant__ CUtensorMap tmap, int* __restrict__ err)
{
    step_tile<kMode, kTma>(d, src, dst, &tmap, err, blockIdx.x, blockIdx.y);
}

// Simulation of block b in a batched launch (first[s] <= b < first[s + 1]).
__device__ __forceinline__ int batch_sim(const BatchArgs& args, int b)
{
    int s = 0;
    while (s + 1 < args.n && b >= args.first[s + 1]) ++s;
    return s;
}

// As batch_sim, with the simulation's parameter block copied to shared
// memory (for the 16-bit kernel, whose register pressure turns every use of
// the indexed kernel-parameter copy into a reload; measured twice as fast).
__device__ __forceinline__ int batch_sim_smem(const BatchArgs& args, int b, LbmDev* s_dev)
{
    const int s = batch_sim(args, b);
    static_assert(sizeof(LbmDev) % 4 == 0 && sizeof(LbmDev) / 4 <= kTileX * kTileY, "LbmDev copy");
    const int tid = threadIdx.y * kTileX + threadIdx.x;
    if (tid < (int)(sizeof(LbmDev) / 4))
        reinterpret_cast<int*>(s_dev)[tid] = reinterpret_cast<const int*>(&args.dev[s])[tid];
    __syncthreads();
    return s;
}

// Many simulations in one launch: block b takes tile b - first[s] of the
// simulation s with first[s] <= b < first[s + 1], tiles numbered row by row.
template <bool kTma>
__global__ void __launch_bounds__(kTileX * kTileY, 4)
    step_batch_kernel(const __grid_constant__ BatchArgs args)
{
    const int s = batch_sim(args, blockIdx.x);
    const int t = blockIdx.x - args.first[s];
    const int tiles_x = (args.dev[s].nx + kTileX - 1) / kTileX;
    step_tile<kStep, kTma>(args.dev[s], static_cast<const float*>(args.src[s]),
                           static_cast<float*>(args.dst[s]),
                           args.has_tmap[s] ? &args.tmap[s] : nullptr, args.err[s],
                           t % tiles_x, t / tiles_x);
}

// Equilibrium populations of set s (0 f, 1 g, 2 h, 3 q) at fluid node (x, y)
// from the macroscopic fields (initial state): P^-1 F(-u) applied to the
// equilibria of Eqs. (26), (31), (37), (42), with n and R from the isotropic
// stencil of phi.
__device__ __forceinline__ void equilibrium_set(const LbmDev& d, const float* __restrict__ fld,
                                                int x, int y, int s, float out[9])
{
    const size_t N = (size_t)d.nx * d.ny;
    const size_t o = (size_t)y * d.nx + x;
    const float phi = fld[o], ux = fld[N + o], uy = fld[2 * N + o], p = fld[3 * N + o];
    const float T = fld[4 * N + o], psi = fld[5 * N + o];
    if (s == 1) {
        const float rho = d.rhoA + __saturatef(phi) * d.drho;
        const float vp = p - rho * kCs2;
        const float ux2 = ux * ux, uy2 = uy * uy;
        central_to_pop(p, -vp * ux, -vp * uy, p * kCs2 + vp * ux2, p * kCs2 + vp * uy2,
                       vp * ux * uy, -vp * (ux2 + kCs2) * uy, -vp * (uy2 + kCs2) * ux,
                       kCs2 * kCs2 * p + vp * (kCs2 * (ux2 + uy2) + ux2 * uy2), ux, uy, out);
        return;
    }
    if (s == 2) {
        scalar_post(T, 0.0f, 0.0f, ux, uy, out);
        return;
    }
    auto phi_at = [&](int xx, int yy) {
        int side;
        const int sy = src_row(d, yy, side);
        return fld[(size_t)sy * d.nx + wrap(xx, d.nx)];
    };
    const float gx = (1.0f / 3.0f) * (phi_at(x + 1, y) - phi_at(x - 1, y)) +
                     (1.0f / 12.0f) * ((phi_at(x + 1, y + 1) - phi_at(x - 1, y + 1)) +
                                       (phi_at(x + 1, y - 1) - phi_at(x - 1, y - 1)));
    const float gy = (1.0f / 3.0f) * (phi_at(x, y + 1) - phi_at(x, y - 1)) +
                     (1.0f / 12.0f) * ((phi_at(x + 1, y + 1) - phi_at(x + 1, y - 1)) +
                                       (phi_at(x - 1, y + 1) - phi_at(x - 1, y - 1)));
    if (s == 0) {
        const float inv = 1.0f / fmaxf(sqrtf(gx * gx + gy * gy), kNormalEps);
        const float theta_m = d.mphi_4_over_W * phi * (1.0f - phi);
        scalar_post(phi, theta_m * gx * inv, theta_m * gy * inv, ux, uy, out);
    } else {
        const float dG = (phi - 0.5f) * (d.g_s32 * phi * (1.0f - phi) + d.g_w);
        const float flux = -d.m_psi * psi * (1.0f - psi) * dG;
        scalar_post(psi, flux * gx, flux * gy, ux, uy, out);
    }
}

__global__ void init_equilibrium_kernel(LbmDev d, const float* __restrict__ fld,
                                        float* __restrict__ pops)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int fy = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= d.nx || fy >= d.nfy) return;
    const int y = d.y0 + fy;
    const size_t N = (size_t)d.nx * d.ny;
    const size_t o = (size_t)y * d.nx + x;
    for (int s = 0; s < 4; ++s) {
        float out[9];
        equilibrium_set(d, fld, x, y, s, out);
#pragma unroll
        for (int a = 0; a < 9; ++a) pops[(size_t)(9 * s + a) * N + o] = out[a];
    }
}

// ---- 16-bit population storage ----------------------------------------------------------
//
// A sim with FP16 or BF16 storage keeps, per node x and set s, the rest state
// m_s(x) = M_s(x)/36 of the populations x pushed at the last step (FP32, one
// float4 (f, g, h, q) per node; M_s the set's zeroth moment), and per
// population its deviation from the lattice-weighted rest state of the node
// that pushed it (16-bit, the set pairs (f, g) and (h, q) side by side,
// [2][9][ny][nx][2], dev_index):
//     f_a(y) = k_a m(src_a(y)) + dev_a(y),   src_a(y) = y - e_a,
// or y itself when y - e_a is a wall row (the population bounced back at y),
// with the integer weights k_a = 36 w_a = 16, 4, 1: k_a m is exact in FP32 and
// the weights sum to 36 exactly, so the conserved scalars are carried without
// the rounding bias that the inexact FP32 weights 4/9, 1/9, 1/36 would add
// every step.  Only the small deviations (velocity, flux and non-equilibrium
// content) are rounded to 16 bits.  m is the post-collision zeroth moment
// over 36 plus the nine deviations' rounding errors over 36, so that the
// populations a node pushes sum to its FP32 values.  All arithmetic is FP32.

// Rest-state moments of a tile plus three nodes of halo, [4][TY + 6][TX + 6];
// slot (mx, my) holds the node at tile-relative (mx - 3, my - 3), wrapped in x
// (and in y without walls); rows past a wall hold mirror values, which are
// never used as population sources.
constexpr int kMW = kTileX + 6, kMH = kTileY + 6;

// Population a of set s shown at M-tile slot (mx, my), physical row py, from
// its deviation dv.
__device__ __forceinline__ float rebuild(const LbmDev& d, const float (*m)[kMH][kMW], int s, int a,
                                         int mx, int my, int py, float dv)
{
    const int ex = ex_dir(a), ey = ey_dir(a);
    const bool bounced = d.walls && (py - ey == 0 || py - ey == d.ny - 1);
    const float ms = bounced ? m[s][my][mx] : m[s][my - ey][mx - ex];
    return fmaf(k_of_dir(a), ms, dv);
}

// Push of one set's populations (the store_set pattern) as deviations from
// k_a m with m = M/36 (M: the set's post-collision zeroth moment); returns the
// rest-state value to record for them, m plus the rounding errors of the nine
// stored deviations over 36, so that they sum to their FP32 values.
// dst_set: the set's first element (dev_index(set, 0, N, 0)); population a of
// node o is element 2 (a N + o) from it.
template <typename S, bool kEnergy>
__device__ __forceinline__ float store_set_dev(S* __restrict__ dst_set, int N, const Nbr& nb,
                                               const float v[9], float M, int wall, float Tw)
{
    // out[a]: the value leaving along a, or, towards a wall, the value that
    // returns to this node in the opposite direction (same weight)
    float out[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) out[a] = v[a];
    if (wall < 0) {
        out[4] = kEnergy ? -v[4] + 2.0f * kW1 * Tw : v[4];
        out[7] = kEnergy ? -v[7] + 2.0f * kW2 * Tw : v[7];
        out[8] = kEnergy ? -v[8] + 2.0f * kW2 * Tw : v[8];
    } else if (wall > 0) {
        out[2] = kEnergy ? -v[2] + 2.0f * kW1 * Tw : v[2];
        out[5] = kEnergy ? -v[5] + 2.0f * kW2 * Tw : v[5];
        out[6] = kEnergy ? -v[6] + 2.0f * kW2 * Tw : v[6];
    }
    S q[9];
    const float m = M * kInv36;
    float lost = 0.0f;  // sum of the rounding errors of the nine deviations
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const float dv = fmaf(-k_of_dir(a), m, out[a]);
        q[a] = f2s<S>(dv);
        lost += dv - s2f<S>(q[a]);
    }
    const int o0 = nb.o[0];
    dst_set[2 * o0] = q[0];
    dst_set[2 * (N + nb.o[1])] = q[1];
    dst_set[2 * (3 * N + nb.o[3])] = q[3];
    if (wall == 0) {
        dst_set[2 * (2 * N + nb.o[2])] = q[2];
        dst_set[2 * (4 * N + nb.o[4])] = q[4];
        dst_set[2 * (5 * N + nb.o[5])] = q[5];
        dst_set[2 * (6 * N + nb.o[6])] = q[6];
        dst_set[2 * (7 * N + nb.o[7])] = q[7];
        dst_set[2 * (8 * N + nb.o[8])] = q[8];
    } else if (wall < 0) {
        dst_set[2 * (2 * N + nb.o[2])] = q[2];
        dst_set[2 * (5 * N + nb.o[5])] = q[5];
        dst_set[2 * (6 * N + nb.o[6])] = q[6];
        dst_set[2 * (2 * N + o0)] = q[4];
        dst_set[2 * (5 * N + o0)] = q[7];
        dst_set[2 * (6 * N + o0)] = q[8];
    } else {
        dst_set[2 * (4 * N + nb.o[4])] = q[4];
        dst_set[2 * (7 * N + nb.o[7])] = q[7];
        dst_set[2 * (8 * N + nb.o[8])] = q[8];
        dst_set[2 * (4 * N + o0)] = q[2];
        dst_set[2 * (7 * N + o0)] = q[5];
        dst_set[2 * (8 * N + o0)] = q[6];
    }
    return fmaf(lost, kInv36, m);
}

// node_update's store for 16-bit storage: deviations pushed to the
// neighbours, the four rest-state moments written at the node.
template <typename S>
struct StoreDev {
    S* dev;
    float4* mom;
    template <bool kEnergy>
    __device__ __forceinline__ float put(int set, int N, const Nbr& nb, const float v[9], float M,
                                         int wall, float Tw) const
    {
        return store_set_dev<S, kEnergy>(dev + dev_index(set, 0, N, 0), N, nb, v, M, wall, Tw);
    }
    __device__ __forceinline__ void finish(int o, float Mf, float Mg, float Mh, float Mq) const
    {
        mom[o] = make_float4(Mf, Mg, Mh, Mq);
    }
};

// The fused step (or, kFields, the field evaluation) of tile (bx, by) of a
// sim with 16-bit storage: the populations are rebuilt in FP32 from the
// deviations and the rest-state moments while they are staged, then the
// update is node_update's.
template <int kMode, typename S>
__device__ __forceinline__ void step_tile_dev(const LbmDev& d, const S* __restrict__ dsrc,
                                              const float4* __restrict__ msrc,
                                              S* __restrict__ ddst, float4* __restrict__ mdst,
                                              float* __restrict__ fdst, int bx, int by)
{
    constexpr int TX = kTileX, TY = kTileY;
    constexpr int EW = TX + 4, EH = TY + 4;
    constexpr int RW = TX + 2, RH = TY + 2;
    extern __shared__ __align__(128) unsigned char s_dyn[];
    float(*s_pop)[TY][TX] = reinterpret_cast<float(*)[TY][TX]>(s_dyn);  // [36][TY][TX]
    __shared__ float s_m[4][kMH][kMW];
    __shared__ float s_phi[EH][EW];
    __shared__ float s_sig[RH][RW];
    __shared__ float s_phs[RH][RW];
    __shared__ float s_nx[RH][RW];
    __shared__ float s_ny[RH][RW];
    const TileSmem sm{s_pop, s_phi, s_sig, s_phs, s_nx, s_ny};

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int x0 = bx * TX;
    const int fy0 = by * TY;
    const int N = d.nx * d.ny;
    const int gx = x0 + tx;
    const int gfy = fy0 + ty;
    const bool active = (gx < d.nx) && (gfy < d.nfy);
    const int gy = d.y0 + gfy;

    for (int i = tid; i < kMW * kMH; i += TX * TY) {
        const int mx = i % kMW, my = i / kMW;
        int side;
        const int sx = wrap_x(d, x0 + mx - 3);
        const int sy = src_row(d, d.y0 + fy0 + my - 3, side);
        const float4 mv = __ldg(msrc + (sy * d.nx + sx));
        s_m[0][my][mx] = mv.x;
        s_m[1][my][mx] = mv.y;
        s_m[2][my][mx] = mv.z;
        s_m[3][my][mx] = mv.w;
    }
    __syncthreads();

    // M-tile row of the node whose populations slot row r (tile-relative,
    // physical row py) shows: the slot's own row, or with walls the row of its
    // mirror source sy; clamped so that slots past a second reflection (which
    // feed only inactive nodes) stay inside the tile.
    auto mrow = [&](int r_slot, int sy) {
        const int r = d.walls ? (sy - d.y0 - fy0) + 3 : r_slot;
        return min(max(r, 1), kMH - 2);
    };

    int own_side = 0;
    {
        const int sx = wrap_x(d, gx);
        const int sy = src_row(d, gy, own_side);
        const int my = mrow(ty + 3, sy);
        const int o = sy * d.nx + sx;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 9; ++a)
                s_pop[9 * s + a][ty][tx] =
                    rebuild(d, s_m, s, a, tx + 3, my, sy, s2f<S>(__ldg(dsrc + dev_index(s, a, N, o))));
    }

    for (int i = tid; i < EW * EH; i += TX * TY) {
        const int ex = i % EW, ey = i / EW;
        if (ex >= 2 && ex < TX + 2 && ey >= 2 && ey < TY + 2) continue;
        const bool ring1 = ex >= 1 && ex <= TX + 2 && ey >= 1 && ey <= TY + 2;
        int side;
        const int sx = wrap_x(d, x0 + ex - 2);
        const int sy = src_row(d, d.y0 + fy0 + ey - 2, side);
        const int my = mrow(ey + 1, sy);
        const int o = sy * d.nx + sx;
        float sums[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const int nsets = ring1 ? 4 : 1;
        for (int s = 0; s < nsets; ++s) {
            float v[9];
#pragma unroll
            for (int a = 0; a < 9; ++a)
                v[a] = rebuild(d, s_m, s, a, ex + 1, my, sy, s2f<S>(__ldg(dsrc + dev_index(s, a, N, o))));
            sums[s] = sum9(v);
        }
        halo_fields(d, sm, ex, ey, ring1, side, sums[0], sums[1], sums[2], sums[3]);
    }

    const OwnPops own{&s_pop[0][ty][tx], TX * TY};
    const NodeMoments m = own_moments(d, sm, own, tx, ty, own_side);
    __syncthreads();
    normals_pass(sm, tid, TX * TY);
    __syncthreads();
    if (!active) return;
    node_update<kMode>(d, sm, m, own, StoreDev<S>{ddst, mdst}, fdst, tx, ty, gx, gy);
}

constexpr int kDevPopSmem = 36 * kTileX * kTileY * sizeof(float);  // dynamic shared memory

template <int kMode, typename S>
__global__ void __launch_bounds__(kTileX * kTileY, 4)
    step_dev_kernel(LbmDev d, const S* __restrict__ dsrc, const float4* __restrict__ msrc,
                    S* __restrict__ ddst, float4* __restrict__ mdst, float* __restrict__ fdst)
{
    step_tile_dev<kMode, S>(d, dsrc, msrc, ddst, mdst, fdst, blockIdx.x, blockIdx.y);
}

template <typename S>
__global__ void __launch_bounds__(kTileX * kTileY, 4)
    step_batch_dev_kernel(const __grid_constant__ BatchArgs args)
{
    __shared__ LbmDev s_dev;
    const int s = batch_sim_smem(args, blockIdx.x, &s_dev);
    const int t = blockIdx.x - args.first[s];
    const int tiles_x = (s_dev.nx + kTileX - 1) / kTileX;
    step_tile_dev<kStep, S>(s_dev, static_cast<const S*>(args.src[s]),
                            static_cast<const float4*>(args.msrc[s]), static_cast<S*>(args.dst[s]),
                            static_cast<float4*>(args.mdst[s]), nullptr, t % tiles_x,
                            t / tiles_x);
}

// Source node of population a at fluid node (x, y) for the rest-state
// reference: y - e_a, or (x, y) itself when y - e_a is a wall row.
__device__ __forceinline__ int src_node(const LbmDev& d, int x, int y, int a)
{
    const int ex = ex_dir(a), ey = ey_dir(a);
    if (d.walls && (y - ey == 0 || y - ey == d.ny - 1)) return y * d.nx + x;
    return wrap(y - ey, d.ny) * d.nx + wrap(x - ex, d.nx);
}

__device__ __forceinline__ float& comp(float4& v, int s)
{
    return s == 0 ? v.x : (s == 1 ? v.y : (s == 2 ? v.z : v.w));
}

// Deviations of populations a0 .. a0 + count - 1 (FP32 planes pl[k][ny][nx])
// from the rest states mom (FP32 populations to 16-bit storage); the
// rounding errors of each node's deviations are summed per set into lost
// (cleared by the call with a0 = 0) for fold_lost_kernel.
template <typename S>
__global__ void split_planes_kernel(LbmDev d, const float* __restrict__ pl, int a0, int count,
                                    const float4* __restrict__ mom, S* __restrict__ dev,
                                    float4* __restrict__ lost)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int fy = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= d.nx || fy >= d.nfy) return;
    const int y = d.y0 + fy;
    const size_t N = (size_t)d.nx * d.ny;
    const int o = y * d.nx + x;
    float4 l = a0 == 0 ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : lost[o];
    for (int k = 0; k < count; ++k) {
        const int a = (a0 + k) % 9, s = (a0 + k) / 9;
        float4 mv = mom[src_node(d, x, y, a)];
        const float dv = fmaf(-k_of_dir(a), comp(mv, s), pl[(size_t)k * N + o]);
        const S q = f2s<S>(dv);
        dev[dev_index(s, a, N, o)] = q;
        comp(l, s) += dv - s2f<S>(q);
    }
    lost[o] = l;
}

// mom += lost / 36 at every fluid node: the populations held at a node then
// sum, over the lattice, to the FP32 values they were split from (each node's
// m is referenced once per direction, with integer weights summing to 36).
__global__ void fold_lost_kernel(LbmDev d, float4* __restrict__ mom,
                                 const float4* __restrict__ lost)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int fy = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= d.nx || fy >= d.nfy) return;
    const int o = (d.y0 + fy) * d.nx + x;
    const float4 m = mom[o], l = lost[o];
    mom[o] = make_float4(fmaf(l.x, kInv36, m.x), fmaf(l.y, kInv36, m.y), fmaf(l.z, kInv36, m.z),
                         fmaf(l.w, kInv36, m.w));
}

// FP32 populations a0 .. a0 + count - 1 rebuilt from 16-bit storage into
// pl[k][ny][nx] (wall rows 0).
template <typename S>
__global__ void join_planes_kernel(LbmDev d, const S* __restrict__ dev,
                                   const float4* __restrict__ mom, int a0, int count,
                                   float* __restrict__ pl)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= d.nx || y >= d.ny) return;
    const size_t N = (size_t)d.nx * d.ny;
    const int o = y * d.nx + x;
    const bool fluid = !d.walls || (y >= 1 && y <= d.ny - 2);
    for (int k = 0; k < count; ++k) {
        const int a = (a0 + k) % 9, s = (a0 + k) / 9;
        float v = 0.0f;
        if (fluid) {
            const float4 mv = mom[src_node(d, x, y, a)];
            const float ms = s == 0 ? mv.x : (s == 1 ? mv.y : (s == 2 ? mv.z : mv.w));
            v = fmaf(k_of_dir(a), ms, s2f<S>(dev[dev_index(s, a, N, o)]));
        }
        pl[(size_t)k * N + o] = v;
    }
}

// Initial state of a sim with 16-bit storage: the equilibria of
// equilibrium_set as deviations from k_a m(src_a), where 36 m = (phi, p, T, psi)
// of the fields (the zeroth moments of the four equilibria).
template <typename S>
__global__ void init_dev_kernel(LbmDev d, const float* __restrict__ fld, S* __restrict__ dev,
                                float4* __restrict__ mom)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int fy = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= d.nx || fy >= d.nfy) return;
    const int y = d.y0 + fy;
    const size_t N = (size_t)d.nx * d.ny;
    const int o = y * d.nx + x;
    constexpr int kField[4] = {0, 3, 4, 5};  // phi, p, T, psi
    float lost[4];  // rounding errors of the node's deviations, folded into its M
    for (int s = 0; s < 4; ++s) {
        float out[9];
        equilibrium_set(d, fld, x, y, s, out);
        lost[s] = 0.0f;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const float ms = fld[(size_t)kField[s] * N + src_node(d, x, y, a)] * kInv36;
            const float dv = fmaf(-k_of_dir(a), ms, out[a]);
            const S q = f2s<S>(dv);
            dev[dev_index(s, a, N, o)] = q;
            lost[s] += dv - s2f<S>(q);
        }
    }
    mom[o] = make_float4(fmaf(lost[0], kInv36, fld[o] * kInv36),
                         fmaf(lost[1], kInv36, fld[3 * N + o] * kInv36),
                         fmaf(lost[2], kInv36, fld[4 * N + o] * kInv36),
                         fmaf(lost[3], kInv36, fld[5 * N + o] * kInv36));
}

// Analytic initial fields: tanh bubble (Sec. 3 profile), fluid at rest, T
// linear between the wall planes, psi uniform (psi0) or, with psi_bc 1 or 2,
// linear from psi_L to psi_R between the wall planes.
__global__ void analytic_fields_kernel(LbmDev d, float* __restrict__ fld)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= d.nx || y >= d.ny) return;
    const size_t N = (size_t)d.nx * d.ny;
    const size_t o = (size_t)y * d.nx + x;
    float phi = 0.0f;
    if (d.R > 0.0f) {
        const float r = hypotf((float)x - d.xb, (float)y - d.yb);
        phi = 0.5f + 0.5f * tanhf(2.0f * (d.R - r) / d.W);
    }
    float T = d.T_ref;
    if (d.walls) T = d.T_H + (d.T_C - d.T_H) * ((float)y - 0.5f) / (float)(d.ny - 2);
    float psi = d.psi0;
    if (d.walls && d.psi_bc != 0)
        psi = d.psi_L + (d.psi_R - d.psi_L) * ((float)y - 0.5f) / (float)(d.ny - 2);
    const bool fluid = !d.walls || (y >= 1 && y <= d.ny - 2);
    fld[o] = fluid ? phi : 0.0f;
    fld[N + o] = 0.0f;
    fld[2 * N + o] = 0.0f;
    fld[3 * N + o] = 0.0f;
    fld[4 * N + o] = fluid ? T : 0.0f;
    fld[5 * N + o] = fluid ? psi : 0.0f;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// FP64 block sums of the observables; fixed grid and order: deterministic.
__global__ void __launch_bounds__(kReduceThreads)
    observe_partial_kernel(LbmDev d, const float* __restrict__ fld, double* __restrict__ part)
{
    constexpr int K = 8;
    double acc[K] = {0, 0, 0, 0, 0, 0, 0, 0};
    const size_t N = (size_t)d.nx * d.ny;
    const long long total = (long long)d.nx * d.nfy;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % d.nx);
        const int y = d.y0 + (int)(i / d.nx);
        const size_t o = (size_t)y * d.nx + x;
        const float phi = fld[o], ux = fld[N + o], uy = fld[2 * N + o], p = fld[3 * N + o];
        const float T = fld[4 * N + o], psi = fld[5 * N + o];
        const bool bad = !(isfinite(phi) && isfinite(ux) && isfinite(uy) && isfinite(p) &&
                           isfinite(T) && isfinite(psi));
        acc[0] += (double)phi;
        acc[1] += (double)psi;
        acc[2] += (double)phi * x;
        acc[3] += (double)phi * y;
        acc[4] += (double)phi * ux;
        acc[5] += (double)phi * uy;
        acc[6] += bad ? 1.0 : 0.0;
        acc[7] += 1.0;
    }
    __shared__ double sm[kReduceThreads / 32][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sm[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) s += sm[w][threadIdx.x];
        part[(size_t)blockIdx.x * K + threadIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kReduceThreads)
    observe_final_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ out)
{
    constexpr int K = 8;
    __shared__ double sm[kReduceThreads / 32][K];
    double acc[K] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += part[(size_t)b * K + k];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sm[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) s += sm[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

dim3 step_grid(const LbmDev& d)
{
    return dim3((d.nx + kTileX - 1) / kTileX, (d.nfy + kTileY - 1) / kTileY);
}

}  // namespace

cudaError_t launch_step(const LbmDev& d, const float* src, float* dst, const CUtensorMap* tmap,
                        int* err, cudaStream_t s)
{
    if (tmap)
        step_kernel<kStep, true><<<step_grid(d), dim3(kTileX, kTileY), 0, s>>>(d, src, dst, *tmap, err);
    else
        step_kernel<kStep, false><<<step_grid(d), dim3(kTileX, kTileY), 0, s>>>(d, src, dst,
                                                                                CUtensorMap{}, err);
    return cudaGetLastError();
}

cudaError_t launch_fields(const LbmDev& d, const float* src, float* fields, const CUtensorMap* tmap,
                          int* err, cudaStream_t s)
{
    if (tmap)
        step_kernel<kFields, true><<<step_grid(d), dim3(kTileX, kTileY), 0, s>>>(d, src, fields,
                                                                                 *tmap, err);
    else
        step_kernel<kFields, false><<<step_grid(d), dim3(kTileX, kTileY), 0, s>>>(
            d, src, fields, CUtensorMap{}, err);
    return cudaGetLastError();
}

int tiles_of(const LbmDev& d)
{
    return ((d.nx + kTileX - 1) / kTileX) * ((d.nfy + kTileY - 1) / kTileY);
}

cudaError_t launch_step_batch(const BatchArgs& args, int total_tiles, cudaStream_t s)
{
    step_batch_kernel<true><<<total_tiles, dim3(kTileX, kTileY), 0, s>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_analytic_fields(const LbmDev& d, float* fields, cudaStream_t s)
{
    dim3 b(32, 8), g((d.nx + 31) / 32, (d.ny + 7) / 8);
    analytic_fields_kernel<<<g, b, 0, s>>>(d, fields);
    return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(const LbmDev& d, const float* fields, float* pops,
                                    cudaStream_t s)
{
    dim3 b(32, 8), g((d.nx + 31) / 32, (d.nfy + 7) / 8);
    init_equilibrium_kernel<<<g, b, 0, s>>>(d, fields, pops);
    return cudaGetLastError();
}

cudaError_t launch_observe_reduce(const LbmDev& d, const float* fields, double* partials,
                                  int nblocks, double* result, cudaStream_t s)
{
    observe_partial_kernel<<<nblocks, kReduceThreads, 0, s>>>(d, fields, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    observe_final_kernel<<<1, kReduceThreads, 0, s>>>(partials, nblocks, result);
    return cudaGetLastError();
}

namespace {

// The 16-bit kernels keep their population tile in dynamic shared memory
// (static + dynamic > 48 KB needs the opt-in).
template <typename S>
cudaError_t allow_dev_smem()
{
    cudaError_t e = cudaFuncSetAttribute(step_dev_kernel<kStep, S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kDevPopSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_dev_kernel<kFields, S>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kDevPopSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_batch_dev_kernel<S>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kDevPopSmem);
    return e;
}

template <typename S>
cudaError_t launch_step_dev_t(const LbmDev& d, const void* dsrc, const float4* msrc, void* ddst,
                              float4* mdst, float* fields, cudaStream_t s)
{
    if (fields)
        step_dev_kernel<kFields, S><<<step_grid(d), dim3(kTileX, kTileY), kDevPopSmem, s>>>(
            d, static_cast<const S*>(dsrc), msrc, nullptr, nullptr, fields);
    else
        step_dev_kernel<kStep, S><<<step_grid(d), dim3(kTileX, kTileY), kDevPopSmem, s>>>(
            d, static_cast<const S*>(dsrc), msrc, static_cast<S*>(ddst), mdst, nullptr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_dev_storage(int precision)
{
    if (precision == LBM_FP16) return allow_dev_smem<__half>();
    if (precision == LBM_BF16) return allow_dev_smem<__nv_bfloat16>();
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_dev(const LbmDev& d, int precision, const void* dsrc, const float4* msrc,
                            void* ddst, float4* mdst, float* fields, cudaStream_t s)
{
    if (precision == LBM_FP16)
        return launch_step_dev_t<__half>(d, dsrc, msrc, ddst, mdst, fields, s);
    if (precision == LBM_BF16)
        return launch_step_dev_t<__nv_bfloat16>(d, dsrc, msrc, ddst, mdst, fields, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_batch_dev(const BatchArgs& args, int precision, int total_tiles,
                                  cudaStream_t s)
{
    if (precision == LBM_FP16)
        step_batch_dev_kernel<__half>
            <<<total_tiles, dim3(kTileX, kTileY), kDevPopSmem, s>>>(args);
    else if (precision == LBM_BF16)
        step_batch_dev_kernel<__nv_bfloat16>
            <<<total_tiles, dim3(kTileX, kTileY), kDevPopSmem, s>>>(args);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_init_dev(const LbmDev& d, int precision, const float* fields, void* dev,
                            float4* mom, cudaStream_t s)
{
    dim3 b(32, 8), g((d.nx + 31) / 32, (d.nfy + 7) / 8);
    if (precision == LBM_FP16)
        init_dev_kernel<__half><<<g, b, 0, s>>>(d, fields, static_cast<__half*>(dev), mom);
    else if (precision == LBM_BF16)
        init_dev_kernel<__nv_bfloat16>
            <<<g, b, 0, s>>>(d, fields, static_cast<__nv_bfloat16*>(dev), mom);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_split_planes(const LbmDev& d, int precision, const float* planes, int a0,
                                int count, const float4* mom, void* dev, float4* lost,
                                cudaStream_t s)
{
    dim3 b(32, 8), g((d.nx + 31) / 32, (d.nfy + 7) / 8);
    if (precision == LBM_FP16)
        split_planes_kernel<__half>
            <<<g, b, 0, s>>>(d, planes, a0, count, mom, static_cast<__half*>(dev), lost);
    else if (precision == LBM_BF16)
        split_planes_kernel<__nv_bfloat16>
            <<<g, b, 0, s>>>(d, planes, a0, count, mom, static_cast<__nv_bfloat16*>(dev), lost);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_fold_lost(const LbmDev& d, float4* mom, const float4* lost, cudaStream_t s)
{
    dim3 b(32, 8), g((d.nx + 31) / 32, (d.nfy + 7) / 8);
    fold_lost_kernel<<<g, b, 0, s>>>(d, mom, lost);
    return cudaGetLastError();
}

cudaError_t launch_join_planes(const LbmDev& d, int precision, const void* dev, const float4* mom,
                               int a0, int count, float* planes, cudaStream_t s)
{
    dim3 b(32, 8), g((d.nx + 31) / 32, (d.ny + 7) / 8);
    if (precision == LBM_FP16)
        join_planes_kernel<__half>
            <<<g, b, 0, s>>>(d, static_cast<const __half*>(dev), mom, a0, count, planes);
    else if (precision == LBM_BF16)
        join_planes_kernel<__nv_bfloat16><<<g, b, 0, s>>>(
            d, static_cast<const __nv_bfloat16*>(dev), mom, a0, count, planes);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

namespace {
// One block waits, with the step kernels' bounded wait, on a barrier that
// expects an arrival nothing makes; flag[0] = 1 if the wait gave up.
__global__ void bounded_wait_probe_kernel(uint64_t limit_ns, int* flag)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) mbar_init(b, 1);
    __syncthreads();
    const bool ok = mbar_wait_bounded(b, 0, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) *flag = 1;
}
}  // namespace

cudaError_t launch_bounded_wait_probe(uint64_t limit_ns, int* flag, cudaStream_t s)
{
    bounded_wait_probe_kernel<<<1, 32, 0, s>>>(limit_ns, flag);
    return cudaGetLastError();
}
