// The streaming kernels for one tile shape: this file is included once per
// shape inside a namespace that defines TX (columns of a block, up to 64) and
// TY (rows of a chunk), with the headers lbm_internal.h and lbm_device.cuh
// already included; LBM_STREAM_16BIT (0 or 1) says whether the shape has the
// 16-bit storage kernels.
namespace {

constexpr int NT = TX * TY;       // threads per block, one node each
// Side nodes of a chunk: phi at the outer columns -2 and w + 1, all four
// zeroth moments at the inner columns -1 and w: six items per row, (phi),
// (phi, p*) or (T, psi), taken by the last 6 TY threads of the block.
constexpr int kSideItems = 6 * TY;
// 16-bit storage: rest-moment groups of eight columns, eight on each side
constexpr int kMomGroups = (TX + 16) / 8;
// Window rows: a power of two, at least the 2 TY + 7 rows an iteration's
// update reads (from Y - 4) and the next iteration writes (up to Y + 2 TY - 1
// and the wall mirrors three rows beyond), so that an iteration ends without
// a barrier
constexpr int kSlots = 2 * TY + 7 <= 16 ? 16 : 32;
static_assert(2 * TY + 7 <= kSlots && TX % 8 == 0 && NT == 256, "stream tile shape");

// one-dimensional rest populations E_i(0): 1/6, 2/3, 1/6 at e = -1, 0, +1
__device__ __forceinline__ constexpr float e0_of(int i) { return i == 1 ? 2.0f / 3.0f : 1.0f / 6.0f; }
__device__ __forceinline__ constexpr int opp_dir(int a)
{
    return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5);
}

// ---- moments -----------------------------------------------------------------------------

// The moments of one set.  The zeroth moment is carried as 36 r + d: r a
// reference (FP32: the rest population / 16; 16-bit: the node's own m) and d
// the sum of the small differences t_a = f_a - k_a r, which near equilibrium
// are exact (k_a r is exact and close to f_a), so the conserved scalars are
// not rounded to the precision of their full size at every step; the first
// moments are sums of the same differences (sum_a e_a k_a = 0).
struct SetMom {
    float r, d, jx, jy;
    __device__ __forceinline__ float s() const { return fmaf(36.0f, r, d); }
};

struct Mom {
    SetMom f, g, h, q;
    float gnd, gxy;     // g: sum g (ex^2 - ey^2), sum g ex ey
};

// The sum of one set's differences t[9] (fixed summation order, shared by
// every place that evaluates a node).
__device__ __forceinline__ float sum_t(const float t[9])
{
    return (((t[1] + t[2]) + (t[3] + t[4])) + ((t[5] + t[6]) + (t[7] + t[8]))) + t[0];
}

// FP32 populations f[9] of one set: r = f_0 / 16.
__device__ __forceinline__ float diffs32(const float f[9], float t[9])
{
    const float r = f[0] * 0.0625f;
#pragma unroll
    for (int a = 0; a < 9; ++a) t[a] = fmaf(-k_of_dir(a), r, f[a]);
    return r;
}

// The same sums over packed pairs of sets (one lane per set).
__device__ __forceinline__ float2 sum_t2(const float2 t[9])
{
    return add2(add2(add2(add2(t[1], t[2]), add2(t[3], t[4])), add2(add2(t[5], t[6]), add2(t[7], t[8]))),
                t[0]);
}
__device__ __forceinline__ float2 mx9_2(const float2 v[9])
{
    return add2(add2(sub2(v[1], v[3]), sub2(v[5], v[6])), sub2(v[8], v[7]));
}
__device__ __forceinline__ float2 my9_2(const float2 v[9])
{
    return sub2(add2(sub2(v[2], v[4]), add2(v[5], v[6])), add2(v[7], v[8]));
}

// The moments of a node's FP32 populations get(0 .. 35), sets in the packed
// pairs (f, g) and (h, q): per lane r = f_0/16 and t_a as diffs32, d = sum_t,
// j = (mx9, my9) of t.
template <class Get>
__device__ __forceinline__ Mom moments_of(const Get& get)
{
    Mom m;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        float2 v[9], t[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = make_float2(get(18 * p + a), get(18 * p + 9 + a));
        const float2 r = mul2(v[0], f2(0.0625f));
#pragma unroll
        for (int a = 0; a < 9; ++a) t[a] = fma2(f2(-k_of_dir(a)), r, v[a]);
        const float2 d = sum_t2(t), jx = mx9_2(t), jy = my9_2(t);
        (p ? m.h : m.f) = SetMom{r.x, d.x, jx.x, jy.x};
        (p ? m.q : m.g) = SetMom{r.y, d.y, jx.y, jy.y};
        if (p == 0) {
            m.gnd = (t[1].y + t[3].y) - (t[2].y + t[4].y);
            m.gxy = (t[5].y + t[7].y) - (t[6].y + t[8].y);
        }
    }
    return m;
}

// ---- one-dimensional factors of the inverse frame change -------------------------------

struct Axis {
    float dE[3], E[3], Z[3], O[3];  // index 0: e = -1, 1: e = 0, 2: e = +1
};

__device__ __forceinline__ Axis axis_of(float u)
{
    Axis A;
    const float u2 = u * u;
    A.dE[0] = 0.5f * (u2 - u);
    A.dE[1] = -u2;
    A.dE[2] = 0.5f * (u2 + u);
#pragma unroll
    for (int i = 0; i < 3; ++i) A.E[i] = e0_of(i) + A.dE[i];
    A.Z[0] = A.dE[0];
    A.Z[1] = 1.0f - u2;
    A.Z[2] = A.dE[2];
    A.O[0] = u - 0.5f;
    A.O[1] = -2.0f * u;
    A.O[2] = u + 0.5f;
    return A;
}

// Deviation of direction a of a scalar scheme from its rest value w_a s:
// s (E E - w) + A O Z + B Z O, with E E - w = dE_i E_j + E_i(0) dE_j exactly.
template <int a>
__device__ __forceinline__ float scalar_dev(const Axis& X, const Axis& Y, float s, float A, float B)
{
    constexpr int i = ex_dir(a) + 1, j = ey_dir(a) + 1;
    const float D = fmaf(X.dE[i], Y.E[j], e0_of(i) * Y.dE[j]);
    return fmaf(s, D, fmaf(A, X.O[i] * Y.Z[j], B * (X.Z[i] * Y.O[j])));
}

// ---- the circular field window ----------------------------------------------------------

// Row r of the lattice (unwrapped numbering along the strip) sits in slot
// r & (SLOTS - 1).  phi carries two columns of halo (column c at c + 2), the
// others one (c + 1).
template <int SLOTS>
struct Window {
    float phi[SLOTS][TX + 4];
    float sig[SLOTS][TX + 2];
    float phs[SLOTS][TX + 2];
    float nrx[SLOTS][TX + 2];
    float nry[SLOTS][TX + 2];
    // moments of a chunk's top two rows, updated one iteration later; each
    // slot is written and read by the same thread
    Mom carry[2][TX];
};

// Isotropic gradient 3 sum_a w_a e_a X(x + e_a) from three rows.
__device__ __forceinline__ void grad_rows(const float* __restrict__ rm, const float* __restrict__ r0,
                                          const float* __restrict__ rp, int c, float& gx, float& gy)
{
    const float e = r0[c + 1], w = r0[c - 1], n = rp[c], s = rm[c];
    const float ne = rp[c + 1], nw = rp[c - 1], se = rm[c + 1], sw = rm[c - 1];
    gx = (1.0f / 3.0f) * (e - w) + (1.0f / 12.0f) * ((ne - nw) + (se - sw));
    gy = (1.0f / 3.0f) * (n - s) + (1.0f / 12.0f) * ((ne - se) + (nw - sw));
}

// Fields of one node into window row r (phys: its physical row) at local
// column c, and the mirror rows a wall makes of it: rows 1, 2 mirror to 0, -1
// and rows ny-2, ny-3 to ny-1, ny (phi everywhere, p* - rho c_s^2 and sigma on
// the first mirror row, sigma from 2 T_w - T and the psi ghost).  Rows beyond
// the top wall carry no fields of their own.
template <int SLOTS>
__device__ __forceinline__ void put_fields(const LbmDev& d, Window<SLOTS>& W, int r, int phys, int c,
                                           float phi, float pst, float T, float psi, bool inner)
{
    constexpr int M = SLOTS - 1;
    if (d.walls && phys > d.ny - 2) return;
    W.phi[r & M][c + 2] = phi;
    const float phs = pst - (d.rhoA + __saturatef(phi) * d.drho) * kCs2;
    float sg = 0.0f;
    if (inner) {
        sg = sigma_eos(d, T, psi);
        W.phs[r & M][c + 1] = phs;
        W.sig[r & M][c + 1] = sg;
    }
    if (!d.walls) return;
    if (phys == 1 || phys == d.ny - 2) {
        const int side = phys == 1 ? -1 : 1;
        const int rm = r + side;
        W.phi[rm & M][c + 2] = phi;
        if (inner) {
            W.phs[rm & M][c + 1] = phs;
            W.sig[rm & M][c + 1] =
                sigma_eos(d, 2.0f * (side < 0 ? d.T_H : d.T_C) - T, psi_ghost(d, psi, side));
        }
    }
    if (phys == 2) W.phi[(r - 3) & M][c + 2] = phi;
    if (phys == d.ny - 3) W.phi[(r + 3) & M][c + 2] = phi;
}

// phi of a side node (column c, window row r, physical row phys) and its
// wall mirrors, as put_fields.
template <int SLOTS>
__device__ __forceinline__ void put_side_phi(const LbmDev& d, Window<SLOTS>& W, int r, int phys,
                                             int c, float phi)
{
    constexpr int M = SLOTS - 1;
    if (d.walls && phys > d.ny - 2) return;
    W.phi[r & M][c + 2] = phi;
    if (!d.walls) return;
    if (phys == 1) W.phi[(r - 1) & M][c + 2] = phi;
    if (phys == d.ny - 2) W.phi[(r + 1) & M][c + 2] = phi;
    if (phys == 2) W.phi[(r - 3) & M][c + 2] = phi;
    if (phys == d.ny - 3) W.phi[(r + 3) & M][c + 2] = phi;
}

// phi and p* - rho c_s^2 (what = 1; a0 = phi, a1 = p*) or sigma (what = 2;
// a0 = T, a1 = psi) of an inner side node and their wall mirrors, as
// put_fields.
template <int SLOTS>
__device__ __forceinline__ void put_side_pair(const LbmDev& d, Window<SLOTS>& W, int r, int phys,
                                              int c, int what, float a0, float a1)
{
    constexpr int M = SLOTS - 1;
    if (what == 1) put_side_phi(d, W, r, phys, c, a0);
    if (d.walls && phys > d.ny - 2) return;
    const bool mir = d.walls && (phys == 1 || phys == d.ny - 2);
    const int side = phys == 1 ? -1 : 1;
    const int rm = r + side;
    if (what == 1) {
        const float phs = a1 - (d.rhoA + __saturatef(a0) * d.drho) * kCs2;
        W.phs[r & M][c + 1] = phs;
        if (mir) W.phs[rm & M][c + 1] = phs;
    } else {
        W.sig[r & M][c + 1] = sigma_eos(d, a0, a1);
        if (mir)
            W.sig[rm & M][c + 1] =
                sigma_eos(d, 2.0f * (side < 0 ? d.T_H : d.T_C) - a0, psi_ghost(d, a1, side));
    }
}

// Unit normals n = grad phi / max(|grad phi|, eps) of window rows r0 .. r0 + 7.
template <int SLOTS>
__device__ __forceinline__ void normals_rows(Window<SLOTS>& W, int r0, int tid)
{
    constexpr int M = SLOTS - 1, RW = TX + 2;
    for (int i = tid; i < TY * RW; i += NT) {
        const int r = r0 + i / RW, c = i % RW;
        float gx, gy;
        grad_rows(W.phi[(r - 1) & M], W.phi[r & M], W.phi[(r + 1) & M], c + 1, gx, gy);
        const float inv = fminf(rsqrtf(gx * gx + gy * gy), 1.0f / kNormalEps);
        W.nrx[r & M][c] = gx * inv;
        W.nry[r & M][c] = gy * inv;
    }
}

// ---- destinations of the push ----------------------------------------------------------

// Plane offsets of the nine destinations of node (x, y): periodic x, and
// periodic y without walls.  With walls, directions into a wall return to
// the node (halfway bounce-back) in the opposite direction's plane.
struct Dest {
    int o[9];
    int wall;  // -1 bottom fluid row, +1 top fluid row, 0 otherwise
};

__device__ __forceinline__ Dest dest_of(const LbmDev& d, int x, int y)
{
    const int xw = (x == 0) ? d.nx - 1 : x - 1;
    const int xe = (x + 1 == d.nx) ? 0 : x + 1;
    const int r = y * d.nx;
    int rs = r - d.nx, rn = r + d.nx;
    if (!d.walls) {
        if (y == 0) rs = (d.ny - 1) * d.nx;
        if (y == d.ny - 1) rn = 0;
    }
    Dest D;
    D.o[0] = r + x;
    D.o[1] = r + xe;
    D.o[2] = rn + x;
    D.o[3] = r + xw;
    D.o[4] = rs + x;
    D.o[5] = rn + xe;
    D.o[6] = rn + xw;
    D.o[7] = rs + xw;
    D.o[8] = rs + xe;
    D.wall = !d.walls ? 0 : (y == 1 ? -1 : (y == d.ny - 2 ? 1 : 0));
    return D;
}

// Whether direction a leaves through the wall of this row.
__device__ __forceinline__ bool into_wall(int a, int wall)
{
    return (wall < 0 && ey_dir(a) < 0) || (wall > 0 && ey_dir(a) > 0);
}

// ---- storage policies --------------------------------------------------------------------

// FP32 populations pushed to the neighbours.
struct Out32 {
    static constexpr bool kPairs = false;
    float* dst;
    int N;
    // a scalar scheme with zeroth moment 36 r + d from its deviations dev_a
    // from w_a (36 r + d): v_a = k_a r + (k_a d / 36 + dev_a), with the integer
    // weights k_a = 36 w_a (16, 4, 1) and k_a r exact.  The nine values sum to
    // 36 r + d up to one rounding each, a uniform equilibrium maps to itself
    // exactly, and the inexact FP32 weights add no systematic error.
    __device__ __forceinline__ void scalar(int set, const Dest& D, const SetMom& m,
                                           const float dev[9], bool dirichlet, float Tw) const
    {
        const float d36 = m.d * kInv36;
        float v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = fmaf(k_of_dir(a), m.r, fmaf(k_of_dir(a), d36, dev[a]));
        put(set, D, v, dirichlet, Tw);
    }
    __device__ __forceinline__ void general(int set, const Dest& D, float, const float v[9]) const
    {
        put(set, D, v, false, 0.0f);
    }
    __device__ __forceinline__ void put(int set, const Dest& D, const float v[9], bool dirichlet,
                                        float Tw) const
    {
        float* p = dst + (size_t)set * 9 * N;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            if (into_wall(a, D.wall)) {
                const float val = dirichlet ? -v[a] + 2.0f * w_of_dir(a) * Tw : v[a];
                p[opp_dir(a) * N + D.o[0]] = val;
            } else {
                p[a * N + D.o[a]] = v[a];
            }
        }
    }
    __device__ __forceinline__ void finish(const Dest&) const {}
};

// 16-bit deviations from k_a m pushed to the neighbours (m the new rest
// value, close to M/36 for M the set's post-collision zeroth moment; integer
// weights k_a = 16, 4, 1, see lbm_kernels.cu), and at the node its rest value
// m + (M - 36 m - sum of the nine stored deviations)/36, so that the nine
// pushed populations rebuild (k_a m + stored deviation) to exactly M, whatever
// the rounding of the deviations themselves.  The sets are stored in pairs,
// (f, g) and (h, q), one 32-bit word per population and pair: the first set
// of a pair to be computed (g, h: kPairs orders update_node's collisions
// g, f, h, q) is held until the second, and each word is rounded, stored
// and summed for the rest values in one step.
template <typename S>
struct Out16 {
    static constexpr bool kPairs = true;
    uint32_t* dst;
    float4* mdst;
    int N;
    mutable float M[4];
    mutable float held[9], held_m, held_target;   // the pair's first set
    // scalar scheme, zeroth moment 36 r + d conserved: m = r + d/36 and the
    // residue 36 r + d - 36 m (exact) goes to the rest population
    __device__ __forceinline__ void scalar(int set, const Dest& D, const SetMom& ms,
                                           const float dev_in[9], bool dirichlet, float Tw) const
    {
        const float m = fmaf(ms.d, kInv36, ms.r);
        const float target = fmaf(36.0f, ms.r - m, ms.d);
        float dev[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) dev[a] = dev_in[a];
        dev[0] += target;
        store(set, D, m, target, dev, dirichlet, Tw);
    }
    __device__ __forceinline__ void general(int set, const Dest& D, float Mset, const float v[9]) const
    {
        const float m = Mset * kInv36;
        float dev[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) dev[a] = fmaf(-k_of_dir(a), m, v[a]);
        store(set, D, m, fmaf(-36.0f, m, Mset), dev, false, 0.0f);
    }
    // dev: deviations from k_a m summing to target.  A Dirichlet reflection
    // -v + 2 w Tw of v = k m + dev stores the deviation -dev + 2 k (Tw/36 - m)
    // and moves the target by its change.
    __device__ __forceinline__ void store(int set, const Dest& D, float m, float target,
                                          const float dev[9], bool dirichlet, float Tw) const
    {
        float dv[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            dv[a] = dev[a];
            if (into_wall(a, D.wall) && dirichlet) {
                const float out = fmaf(2.0f * k_of_dir(a), fmaf(Tw, kInv36, -m), -dv[a]);
                target += out - dv[a];
                dv[a] = out;
            }
        }
        if (set == 1 || set == 2) {   // first of its pair: hold
#pragma unroll
            for (int a = 0; a < 9; ++a) held[a] = dv[a];
            held_m = m;
            held_target = target;
            return;
        }
        // set 0 completes (f, g), set 3 completes (h, q)
        const int pr = set >> 1;
        float lo[9], hi[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            lo[a] = pr == 0 ? dv[a] : held[a];
            hi[a] = pr == 0 ? held[a] : dv[a];
        }
        uint32_t* p = dst + (size_t)pr * 9 * N;
        float2 stored = f2(0.0f);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const bool wl = into_wall(a, D.wall);
            const uint32_t w = f2s2<S>(lo[a], hi[a]);
            stored = add2(stored, s2f2<S>(w));
            p[(wl ? opp_dir(a) : a) * N + (wl ? D.o[0] : D.o[a])] = w;
        }
        const float m_lo = pr == 0 ? m : held_m, m_hi = pr == 0 ? held_m : m;
        const float t_lo = pr == 0 ? target : held_target, t_hi = pr == 0 ? held_target : target;
        M[2 * pr] = fmaf(t_lo - stored.x, kInv36, m_lo);
        M[2 * pr + 1] = fmaf(t_hi - stored.y, kInv36, m_hi);
    }
    __device__ __forceinline__ void finish(const Dest& D) const
    {
        mdst[D.o[0]] = make_float4(M[0], M[1], M[2], M[3]);
    }
};

// ---- the node update ----------------------------------------------------------------------

// Stencils, forces, velocity and pressure (Sec. 3, App. C; as the tile
// kernels), then the four collisions in moment form and the push.  c: local
// column; r: window row of the node (unwrapped); (x, y): physical node.
template <int SLOTS, class Out>
__device__ __forceinline__ void update_node(const LbmDev& d, const Window<SLOTS>& W, const Mom& m,
                                            int c, int r, int x, int y, const Out& out)
{
    constexpr int K = SLOTS - 1;
    const float* pm = W.phi[(r - 1) & K];
    const float* p0 = W.phi[r & K];
    const float* pp = W.phi[(r + 1) & K];
    float gpx, gpy;
    grad_rows(pm, p0, pp, c + 2, gpx, gpy);
    const float g2 = gpx * gpx + gpy * gpy;
    const float n_x = W.nrx[r & K][c + 1], n_y = W.nry[r & K][c + 1];
    float dnx_dx, dnx_dy, dny_dx, dny_dy;
    grad_rows(W.nrx[(r - 1) & K], W.nrx[r & K], W.nrx[(r + 1) & K], c + 1, dnx_dx, dnx_dy);
    grad_rows(W.nry[(r - 1) & K], W.nry[r & K], W.nry[(r + 1) & K], c + 1, dny_dx, dny_dy);
    const float kappa = dnx_dx + dny_dy;
    float sgx, sgy, phx, phy;
    grad_rows(W.sig[(r - 1) & K], W.sig[r & K], W.sig[(r + 1) & K], c + 1, sgx, sgy);
    grad_rows(W.phs[(r - 1) & K], W.phs[r & K], W.phs[(r + 1) & K], c + 1, phx, phy);
    const float sig = W.sig[r & K][c + 1];
    const float ndots = n_x * sgx + n_y * sgy;
    const float deltas = d.deltas_coef * g2;
    const float phi = m.f.s();
    const float pc = __saturatef(phi);
    const float rho = d.rhoA + pc * d.drho;
    const float inv_rho = __fdividef(1.0f, rho);
    const float Ftx = deltas * (-sig * kappa * n_x + sgx - n_x * ndots) + d.Fext_x;
    const float Fty = deltas * (-sig * kappa * n_y + sgy - n_y * ndots) + d.Fext_y -
                      (rho - d.rhoA) * d.gravity;
    const float Fpx = -phx, Fpy = -phy;
    const float pst = m.g.s();
    const float ux = (3.0f * m.g.jx + 0.5f * Ftx) * inv_rho;
    const float uy = (3.0f * m.g.jy + 0.5f * Fty) * inv_rho;
    const float Gam = Fpx * ux + Fpy * uy;
    const float p = pst + 0.5f * Gam;

    const Dest D = dest_of(d, x, y);
    const Axis X = axis_of(ux), Y = axis_of(uy);

    // ---- f: conservative Allen-Cahn (App. B, Eqs. (26)-(27)) ------------------------------
    const auto collide_f = [&]() {
        const float theta_m = d.mphi_4_over_W * phi * (1.0f - phi);   // M_phi theta
        const float c10 = m.f.jx - ux * phi, c01 = m.f.jy - uy * phi;
        const float A = c10 + d.omega_phi * (theta_m * n_x - c10);
        const float B = c01 + d.omega_phi * (theta_m * n_y - c01);
        float dev[9];
        dev[0] = scalar_dev<0>(X, Y, phi, A, B);
        dev[1] = scalar_dev<1>(X, Y, phi, A, B);
        dev[2] = scalar_dev<2>(X, Y, phi, A, B);
        dev[3] = scalar_dev<3>(X, Y, phi, A, B);
        dev[4] = scalar_dev<4>(X, Y, phi, A, B);
        dev[5] = scalar_dev<5>(X, Y, phi, A, B);
        dev[6] = scalar_dev<6>(X, Y, phi, A, B);
        dev[7] = scalar_dev<7>(X, Y, phi, A, B);
        dev[8] = scalar_dev<8>(X, Y, phi, A, B);
        out.scalar(0, D, m.f, dev, false, 0.0f);
    };
    // ---- h: energy (App. D, Eqs. (37)-(38)), rate from the local diffusivity ----------------
    const auto collide_h = [&]() {
        const float alpha = d.alphaA + pc * d.dalpha;
        const float wT = __fdividef(1.0f, 3.0f * alpha + 0.5f);
        const float T = m.h.s();
        const float c10 = m.h.jx - ux * T, c01 = m.h.jy - uy * T;
        const float A = c10 - wT * c10, B = c01 - wT * c01;
        float dev[9];
        dev[0] = scalar_dev<0>(X, Y, T, A, B);
        dev[1] = scalar_dev<1>(X, Y, T, A, B);
        dev[2] = scalar_dev<2>(X, Y, T, A, B);
        dev[3] = scalar_dev<3>(X, Y, T, A, B);
        dev[4] = scalar_dev<4>(X, Y, T, A, B);
        dev[5] = scalar_dev<5>(X, Y, T, A, B);
        dev[6] = scalar_dev<6>(X, Y, T, A, B);
        dev[7] = scalar_dev<7>(X, Y, T, A, B);
        dev[8] = scalar_dev<8>(X, Y, T, A, B);
        out.scalar(2, D, m.h, dev, true, D.wall < 0 ? d.T_H : d.T_C);
    };
    // ---- q: surfactant (App. E, Eqs. (42)-(43)) -------------------------------------------
    const auto collide_q = [&]() {
        const float psi = m.q.s();
        const float dG = (phi - 0.5f) * (d.g_s32 * phi * (1.0f - phi) + d.g_w);
        const float flux = -d.m_psi * psi * (1.0f - psi) * dG;   // times grad phi
        const float c10 = m.q.jx - ux * psi, c01 = m.q.jy - uy * psi;
        const float A = c10 + d.omega_psi * (flux * gpx - c10);
        const float B = c01 + d.omega_psi * (flux * gpy - c01);
        float dev[9];
        dev[0] = scalar_dev<0>(X, Y, psi, A, B);
        dev[1] = scalar_dev<1>(X, Y, psi, A, B);
        dev[2] = scalar_dev<2>(X, Y, psi, A, B);
        dev[3] = scalar_dev<3>(X, Y, psi, A, B);
        dev[4] = scalar_dev<4>(X, Y, psi, A, B);
        dev[5] = scalar_dev<5>(X, Y, psi, A, B);
        dev[6] = scalar_dev<6>(X, Y, psi, A, B);
        dev[7] = scalar_dev<7>(X, Y, psi, A, B);
        dev[8] = scalar_dev<8>(X, Y, psi, A, B);
        // walls: halfway bounce-back, or anti-bounce-back with psi_L / psi_R
        out.scalar(3, D, m.q, dev, d.psi_bc == 1, D.wall < 0 ? d.psi_L : d.psi_R);
    };
    // ---- g: two-fluid pressure/velocity (App. C, Eqs. (31)-(34)) ----------------------------
    const auto collide_g = [&]() {
        const float mu = d.muA + pc * d.dmu;
        const float wn = __fdividef(1.0f, 3.0f * mu * inv_rho + 0.5f);
        const float vp = p - rho * kCs2;                      // varphi = p - rho c_s^2
        const float ux2 = ux * ux, uy2 = uy * uy;
        // pre-collision central moments the relaxation keeps (rate != 1)
        const float c10 = m.g.jx - ux * pst, c01 = m.g.jy - uy * pst;
        const float c2d = m.gnd - 2.0f * (ux * m.g.jx - uy * m.g.jy) + (ux2 - uy2) * pst;
        const float c11 = m.gxy - ux * m.g.jy - uy * m.g.jx + ux * uy * pst;
        // equilibria (Eq. (31)) and sources (Eq. (32))
        const float e20 = p * kCs2 + vp * ux2, e02 = p * kCs2 + vp * uy2;
        const float e11 = vp * ux * uy;
        const float e21 = -vp * (ux2 + kCs2) * uy;
        const float e12 = -vp * (uy2 + kCs2) * ux;
        // c_s^6 rho + varphi (u_x^2 + c_s^2)(u_y^2 + c_s^2) with its two O(rho)
        // terms cancelled exactly
        const float e22 = kCs2 * kCs2 * p + vp * (kCs2 * (ux2 + uy2) + ux2 * uy2);
        const float s10 = kCs2 * Ftx - ux * Gam, s01 = kCs2 * Fty - uy * Gam;
        const float s20 = 2.0f * kCs2 * Fpx * ux + (ux2 + kCs2) * Gam;
        const float s02 = 2.0f * kCs2 * Fpy * uy + (uy2 + kCs2) * Gam;
        const float s11 = kCs2 * (Fpx * uy + Fpy * ux) + ux * uy * Gam;
        // relaxation (Eq. (33)): rate 1 for 00, 10, 01, 2s, 21, 12, 22 (new value
        // equilibrium + source/2; for 00, 10, 01 that is the old value plus the
        // source, by the definitions of p and u, Eq. (34)), omega_nu for 2d, 11
        const float n00 = pst + Gam;
        const float n10 = c10 + s10, n01 = c01 + s01;
        const float n2s = (e20 + e02) + 0.5f * (s20 + s02);
        const float n2d = c2d + wn * ((e20 - e02) - c2d) + (1.0f - 0.5f * wn) * (s20 - s02);
        const float n11 = c11 + wn * (e11 - c11) + (1.0f - 0.5f * wn) * s11;
        float v[9];
        central_to_pop(n00, n10, n01, 0.5f * (n2s + n2d), 0.5f * (n2s - n2d), n11, e21, e12, e22,
                       ux, uy, v);
        out.general(1, D, n00, v);
    };
    // 16-bit storage writes the sets in pairs (f, g), (h, q), each pair's
    // second set completing it
    if constexpr (Out::kPairs) {
        collide_g();
        collide_f();
        collide_h();
        collide_q();
    } else {
        collide_f();
        collide_h();
        collide_q();
        collide_g();
    }
    out.finish(D);
}

// ---- the strip walk -------------------------------------------------------------------------

// Column geometry of block-local index lb: column lb % ncol of width w
// (TX, or less for the last column of a lattice whose nx is not a
// multiple of TX), strip lb / ncol.
struct Strip {
    int x0, w, c0, c1, nchunks, kfirst, klast;
};

__device__ __forceinline__ Strip strip_of(const LbmDev& d, int strip_chunks, int lb)
{
    Strip s;
    const int ncol = (d.nx + TX - 1) / TX;
    s.x0 = (lb % ncol) * TX;
    s.w = min(TX, d.nx - s.x0);
    s.nchunks = (d.nfy + TY - 1) / TY;
    s.c0 = (lb / ncol) * strip_chunks;
    s.c1 = min(s.c0 + strip_chunks, s.nchunks);
    if (d.walls) {
        // the chunk below is read only for its fields and its top two rows
        // (whose update this strip owns); the last strip ends with an
        // iteration that has no chunk and updates the final two rows
        s.kfirst = s.c0 > 0 ? s.c0 - 1 : 0;
        s.klast = s.c1 == s.nchunks ? s.c1 : s.c1 - 1;
    } else {
        // periodic y (nfy a multiple of 8): the chunk below wraps; the top
        // two rows of the last chunk belong to the first strip
        s.kfirst = s.c0 - 1;
        s.klast = s.c1 - 1;
    }
    return s;
}

__device__ __forceinline__ int chunk_row(const LbmDev& d, const Strip& s, int k)
{
    const int kk = k < 0 ? k + s.nchunks : k;
    return d.y0 + kk * TY;
}

__device__ __forceinline__ int phys_row(const LbmDev& d, int r)
{
    if (d.walls) return r;
    return r < 0 ? r + d.ny : (r >= d.ny ? r - d.ny : r);
}

#if LBM_WALK_LAG
// A node's moments parked in shared memory for one iteration, one float per
// thread and component (conflict-free), two buffers by iteration parity.
struct Park {
    float v[2][18][NT];
    __device__ __forceinline__ void put(int par, int tid, const Mom& m)
    {
        const float x[18] = {m.f.r, m.f.d, m.f.jx, m.f.jy, m.g.r, m.g.d, m.g.jx, m.g.jy, m.h.r,
                             m.h.d, m.h.jx, m.h.jy, m.q.r, m.q.d, m.q.jx, m.q.jy, m.gnd, m.gxy};
#pragma unroll
        for (int i = 0; i < 18; ++i) v[par][i][tid] = x[i];
    }
    __device__ __forceinline__ Mom get(int par, int tid) const
    {
        float x[18];
#pragma unroll
        for (int i = 0; i < 18; ++i) x[i] = v[par][i][tid];
        Mom m;
        m.f = SetMom{x[0], x[1], x[2], x[3]};
        m.g = SetMom{x[4], x[5], x[6], x[7]};
        m.h = SetMom{x[8], x[9], x[10], x[11]};
        m.q = SetMom{x[12], x[13], x[14], x[15]};
        m.gnd = x[16];
        m.gxy = x[17];
        return m;
    }
};

#endif

// FP32 storage: the chunk (box {TX, TY, 36}) and four columns on each side
// (boxes {4, TY, 36}) per stage.
template <int S, int SLOTS>
struct Smem32 {
    float pop[S][36][TY][TX];
    float side[S][2][36][TY][4];
    Window<SLOTS> win;
    uint64_t bar[S];
};

// 16-bit storage: the chunk's deviations as 32-bit words of set pairs, (f, g)
// in planes 0 .. 8 and (h, q) in planes 9 .. 17 (box {TX, TY, 18}), eight
// columns on each side (boxes {8, TY, 18}) and the rest-state moments of rows
// -1 .. TY of the chunk in kMomGroups groups of eight columns (boxes
// {4, 8, TY + 2} of the float4 array), group g covering local columns
// 8 g - 8 .. 8 g - 1.
template <typename T16, int S, int SLOTS>
struct Smem16 {
    uint32_t dev[S][18][TY][TX];
    uint32_t side[S][2][18][TY][8];
    float4 mom[S][kMomGroups][TY + 2][8];
    Window<SLOTS> win;
#if LBM_WALK_LAG
    Park park;
#endif
    uint64_t bar[S];
};

// The walk shared by both storage formats.  Stage policies provide:
//   issue(k, st): copies of chunk k into stage st (one thread);
//   bytes: transaction bytes of one stage;
//   own_moments(st, rb, tx, phys): the 14 moments of chunk row rb, column tx;
//   side_item(st, item, r, phys, rw, W): side item 0 .. 5 of chunk row r (items
//     0, 1: phi at columns -2, w + 1; 2..5: (phi, p*) or (T, psi) at columns -1
//     and w);
//   side_slot(it, item, rr): the item and chunk row of the it-th side thread.
template <int S, int SLOTS, class Stage, class Out>
__device__ __forceinline__ void walk(const LbmDev& d, const Strip& sp, Stage& stg, Window<SLOTS>& W,
                                     uint64_t* bars, int* __restrict__ err, const Out& out)
{
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < S; ++i) mbar_init(smem_addr(&bars[i]), 1);
    }
    __syncthreads();
    // last chunk this strip loads
    const int kload = d.walls ? sp.c1 - 1 : sp.klast;
    if (tid == 0) {
        stg.issue(sp.kfirst, 0 % S, smem_addr(&bars[0]));
        if (S == 2 && sp.kfirst + 1 <= kload) stg.issue(sp.kfirst + 1, 1, smem_addr(&bars[1 % S]));
    }
    uint32_t parity = 0;
    const int rb = (ty + TY - 2) % TY;   // chunk row whose moments this thread computes
    Mom mc{};
    for (int k = sp.kfirst; k <= sp.klast; ++k) {
        const bool have = k <= kload;
        const int st = S == 2 ? (k - sp.kfirst) & 1 : 0;
        const int Y = d.y0 + k * TY;   // unwrapped row of chunk row 0
        bool ok = true;
        if (have) {
            ok = mbar_wait_bounded(smem_addr(&bars[st]), (parity >> st) & 1u);
            parity ^= 1u << st;
            // (a thread whose wait gave up computes from an incomplete stage;
            // only shared memory is written before the check below)
            const int r = Y + rb;
            const int phys = phys_row(d, r);
            if (tx < sp.w) {
                mc = stg.own_moments(st, rb, tx, phys);
                put_fields(d, W, r, phys, tx, mc.f.s(), mc.g.s(), mc.h.s(), mc.q.s(), true);
            }
            if (tid >= NT - kSideItems) {
                int item, rr;
                Stage::side_slot(tid - (NT - kSideItems), item, rr);
                stg.side_item(st, item, rr, phys_row(d, Y + rr), Y + rr, W);
            }
        }
        if (__syncthreads_or(!ok)) {
            // a copy did not arrive in time: report it, and keep the block
            // resident for one more bounded wait on every stage so that no
            // transfer into its shared memory outlives it
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait_bounded(smem_addr(&bars[st]), ((parity >> st) & 1u) ^ 1u);
                if (S == 2 && k + 1 <= kload)
                    mbar_wait_bounded(smem_addr(&bars[st ^ 1]), (parity >> (st ^ 1)) & 1u);
            }
            return;
        }
        // the stage is consumed: refill it
        if (tid == 0) {
            const int kn = k + S;
            if (kn <= kload) stg.issue(kn, st, smem_addr(&bars[st]));
        }
        normals_rows(W, Y - 1, tid);
        __syncthreads();
        if (ty < 2) {
            // the chunk's top two rows (TY - 2, TY - 1) are updated in the
            // next iteration; this one updates those of the previous chunk
            const Mom prev = W.carry[ty][tx];
            if (have) W.carry[ty][tx] = mc;
            mc = prev;
        }
        if (k >= sp.c0) {
            // window row Y - 2 + ty: the previous chunk's top rows (ty < 2) or
            // chunk row ty - 2
            const int r = Y - 2 + ty;
            const int y = phys_row(d, r);
            const bool fluid = !d.walls || (y >= 1 && y <= d.ny - 2);
            if (tx < sp.w && fluid && (ty < 2 || have))
                update_node(d, W, mc, tx, r, sp.x0 + tx, y, out);
        }
        // the next iteration writes rows up to Y + 2 TY + 2 while this one may
        // still read rows from Y - 4: a window of fewer slots needs a barrier
        if (SLOTS < 2 * TY + 7) __syncthreads();
    }
}

#if LBM_WALK_LAG
// The walk with one barrier per chunk.  Iteration k takes chunk k (moments,
// fields, side items) and, in the same phase, the normals of chunk k - 1,
// whose fields the previous iteration's barrier published; after the barrier
// it updates the rows of chunk k - 1 (those walk updates in its iteration
// k - 1), from the moments each thread parked in iteration k - 1 (the top
// two rows' one iteration earlier, through the carry).  Rows written in
// iteration k + 1 before its barrier (fields up to Y + 2 TY + 2, normals from
// Y - 1) and rows read by iteration k's update (from Y - TY - 3) span 3 TY + 6
// rows of the window.  One stage.  The 16-bit kernel, whose warps waited at
// its two barriers for the side columns' rest-moment gathers, runs 5 % faster
// this way; for the FP32 kernel the parked moments cost more than the barrier.
template <int S, int SLOTS, class Stage, class Out>
__device__ __forceinline__ void walk_lag(const LbmDev& d, const Strip& sp, Stage& stg, Window<SLOTS>& W,
                                         Park& park, uint64_t* bars, int* __restrict__ err,
                                         const Out& out)
{
    static_assert(S == 1 && SLOTS >= 3 * TY + 6, "one stage and a window of 3 TY + 6 rows");
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    if (tid == 0) mbar_init(smem_addr(&bars[0]), 1);
    __syncthreads();
    // last chunk this strip loads
    const int kload = d.walls ? sp.c1 - 1 : sp.klast;
    if (tid == 0) stg.issue(sp.kfirst, 0, smem_addr(&bars[0]));
    uint32_t parity = 0;
    const int rb = (ty + TY - 2) % TY;   // chunk row whose moments this thread computes
    for (int k = sp.kfirst; k <= sp.klast + 1; ++k) {
        const bool have = k <= kload;
        const int Y = d.y0 + k * TY;   // unwrapped row of chunk row 0
        bool ok = true;
        if (have) {
            ok = mbar_wait_bounded(smem_addr(&bars[0]), parity);
            parity ^= 1u;
            // (a thread whose wait gave up computes from an incomplete stage;
            // only shared memory is written before the check below)
            const int r = Y + rb;
            const int phys = phys_row(d, r);
            if (tx < sp.w) {
                const Mom mc = stg.own_moments(0, rb, tx, phys);
                put_fields(d, W, r, phys, tx, mc.f.s(), mc.g.s(), mc.h.s(), mc.q.s(), true);
                park.put(k & 1, tid, mc);
            }
            if (tid >= NT - kSideItems) {
                int item, rr;
                Stage::side_slot(tid - (NT - kSideItems), item, rr);
                stg.side_item(0, item, rr, phys_row(d, Y + rr), Y + rr, W);
            }
        }
        if (k > sp.kfirst) normals_rows(W, Y - TY - 1, tid);
        if (__syncthreads_or(!ok)) {
            // a copy did not arrive in time: report it, and keep the block
            // resident for one more bounded wait so that no transfer into its
            // shared memory outlives it
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait_bounded(smem_addr(&bars[0]), parity ^ 1u);
            }
            return;
        }
        // the stage is consumed: refill it
        if (tid == 0 && k + 1 <= kload) stg.issue(k + 1, 0, smem_addr(&bars[0]));
        const int j = k - 1;   // the chunk whose rows this iteration updates
        if (j < sp.kfirst) continue;
        const bool have_j = j <= kload;
        const int Yj = Y - TY;
        Mom m{};
        if (ty < 2) {
            // the chunk's top two rows (TY - 2, TY - 1) are updated one
            // iteration later; this one updates those of chunk j - 1
            m = W.carry[ty][tx];
            if (have_j && tx < sp.w) W.carry[ty][tx] = park.get(j & 1, tid);
        } else if (have_j && tx < sp.w) {
            m = park.get(j & 1, tid);
        }
        if (j >= sp.c0) {
            // window row Yj - 2 + ty: chunk j - 1's top rows (ty < 2) or
            // chunk j's row ty - 2
            const int r = Yj - 2 + ty;
            const int y = phys_row(d, r);
            const bool fluid = !d.walls || (y >= 1 && y <= d.ny - 2);
            if (tx < sp.w && fluid && (ty < 2 || have_j))
                update_node(d, W, m, tx, r, sp.x0 + tx, y, out);
        }
    }
}
#endif

// ---- FP32 stage -------------------------------------------------------------------------

template <int S, int SLOTS>
struct Stage32 {
    Smem32<S, SLOTS>& sm;
    const LbmDev& d;
    const Strip& sp;
    const CUtensorMap* tmap;
    const CUtensorMap* tside;
    static constexpr uint32_t bytes = (36u * TY * TX + 2u * 36u * TY * 4u) * 4u;
    __device__ __forceinline__ void issue(int k, int st, uint32_t bar) const
    {
        const int y = chunk_row(d, sp, k);
        const int xl = sp.x0 == 0 ? d.nx - 4 : sp.x0 - 4;
        const int xr = sp.x0 + sp.w == d.nx ? 0 : sp.x0 + sp.w;
        mbar_expect_tx(bar, bytes);
        tma_load_tile(smem_addr(&sm.pop[st][0][0][0]), tmap, sp.x0, y, bar);
        tma_load_tile(smem_addr(&sm.side[st][0][0][0][0]), tside, xl, y, bar);
        tma_load_tile(smem_addr(&sm.side[st][1][0][0][0]), tside, xr, y, bar);
    }
    __device__ __forceinline__ Mom own_moments(int st, int rb, int tx, int) const
    {
        const float* p = &sm.pop[st][0][rb][tx];
        return moments_of([&](int a) { return p[a * TY * TX]; });
    }
    // item by item, all rows of an item on consecutive threads
    __device__ __forceinline__ static void side_slot(int it, int& item, int& rr)
    {
        item = it / TY;
        rr = it % TY;
    }
    // items 0, 1: phi of the outer columns -2, w + 1; items 2..5: the inner
    // columns -1, w: (phi, p*) or (T, psi)
    template <int SL>
    __device__ __forceinline__ void side_item(int st, int item, int r, int phys, int rw,
                                              Window<SL>& W) const
    {
        const bool outer = item < 2;
        const int lr = outer ? item : (item - 2) / 2;
        const int f = outer ? 0 : (item - 2) % 2;
        const int c = outer ? (lr ? sp.w + 1 : -2) : (lr ? sp.w : -1);
        const int bc = lr ? c - sp.w : c + 4;
        const float* p = &sm.side[st][lr][f * 18][r][bc];
        constexpr int P = TY * 4;
        float v[9], t[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = p[a * P];
        float r0 = diffs32(v, t);
        const float s1 = fmaf(36.0f, r0, sum_t(t));
        if (outer) {
            put_side_phi(d, W, rw, phys, c, s1);
            return;
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = p[(9 + a) * P];
        r0 = diffs32(v, t);
        const float s2 = fmaf(36.0f, r0, sum_t(t));
        put_side_pair(d, W, rw, phys, c, f == 0 ? 1 : 2, s1, s2);
    }
};

// ---- 16-bit stage --------------------------------------------------------------------------

template <typename T16, int S, int SLOTS>
struct Stage16 {
    Smem16<T16, S, SLOTS>& sm;
    const LbmDev& d;
    const Strip& sp;
    const CUtensorMap* tmap;
    const CUtensorMap* tside;
    const CUtensorMap* tmom;
    const float4* msrc;   // rest-state moments of the source buffer (global)
    static constexpr uint32_t bytes =
        (18u * TY * TX + 2u * 18u * TY * 8u) * 4u + kMomGroups * (TY + 2) * 8u * 16u;
    __device__ __forceinline__ void issue(int k, int st, uint32_t bar) const
    {
        const int y = chunk_row(d, sp, k);
        const int xl = sp.x0 == 0 ? d.nx - 8 : sp.x0 - 8;
        const int xr = sp.x0 + sp.w == d.nx ? 0 : sp.x0 + sp.w;
        mbar_expect_tx(bar, bytes);
        tma_load_tile(smem_addr(&sm.dev[st][0][0][0]), tmap, sp.x0, y, bar);
        tma_load_tile(smem_addr(&sm.side[st][0][0][0][0]), tside, xl, y, bar);
        tma_load_tile(smem_addr(&sm.side[st][1][0][0][0]), tside, xr, y, bar);
#pragma unroll
        for (int g = 0; g < kMomGroups; ++g) {
            int x = sp.x0 + 8 * g - 8;
            x = x < 0 ? x + d.nx : (x >= d.nx ? x - d.nx : x);
            tma_load_mom(smem_addr(&sm.mom[st][g][0][0]), tmom, x, y - 1, bar);
        }
    }
    __device__ __forceinline__ static void tma_load_mom(uint32_t dst, const CUtensorMap* map, int x,
                                                        int y, uint32_t bar)
    {
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
            "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(x), "r"(y), "r"(bar)
            : "memory");
    }
    // Rest-state moments in a stage: groups of eight columns, rows -1 .. TY
    // of the chunk.  A node's float4 sits at byte offset own (local column c,
    // -8 <= c < TX + 8; chunk row rr, -1 .. TY); its x neighbours are 16 bytes
    // away within a group and one group minus seven columns away across a
    // group boundary, so the nine sources of a node are three base offsets
    // and immediate row offsets.
    static constexpr int kMomRow = 8 * 16;
    static constexpr int kMomGroup = (TY + 2) * kMomRow;
    struct MomAddr {
        int own, east, west;   // byte offsets of (c, rr), (c + 1, rr), (c - 1, rr)
    };
    __device__ __forceinline__ static MomAddr mom_addr(int c, int rr)
    {
        const int cc = c + 8, i = cc & 7;
        MomAddr m;
        m.own = (cc >> 3) * kMomGroup + (rr + 1) * kMomRow + i * 16;
        m.east = m.own + (i == 7 ? kMomGroup - 7 * 16 : 16);
        m.west = m.own - (i == 0 ? kMomGroup - 7 * 16 : 16);
        return m;
    }
    __device__ __forceinline__ const char* mom_base(int st) const
    {
        return reinterpret_cast<const char*>(&sm.mom[st][0][0][0]);
    }
    // the float4 of the node a population of direction (ex, ey) came from
    template <int ex, int ey>
    __device__ __forceinline__ static float4 mom_src(const char* base, const MomAddr& m)
    {
        const int o = ex > 0 ? m.west : (ex < 0 ? m.east : m.own);
        return *reinterpret_cast<const float4*>(base + o - ey * kMomRow);
    }
    // Sources beyond the lattice's first or last row: next to a wall the
    // population bounced back at the node itself (bounce_lo: the row above the
    // bottom wall, bounce_hi: the row below the top wall); with periodic y the
    // sources of row 0 lie in row ny - 1 and those of row ny - 1 in row 0,
    // outside the stage's rows, and are read from the source buffer (wrap_lo,
    // wrap_hi: those rows, else null; xg: the node's column).
    struct Edge {
        bool bounce_lo = false, bounce_hi = false;
        const float4* wrap_lo = nullptr;
        const float4* wrap_hi = nullptr;
        int xg = 0, nx = 1;
    };
    __device__ __forceinline__ Edge edge_of(int phys, int c) const
    {
        Edge e;
        if (d.walls) {
            e.bounce_lo = phys == 1;
            e.bounce_hi = phys == d.ny - 2;
        } else {
            if (phys == 0) e.wrap_lo = msrc + (size_t)(d.ny - 1) * d.nx;
            if (phys == d.ny - 1) e.wrap_hi = msrc;
        }
        e.xg = sp.x0 + c;
        e.nx = d.nx;
        return e;
    }
    // The differences t_a = f_a - k_a r of a node's populations, r its own rest
    // value: f_a = k_a m(src_a) + dev_a with src_a the node the population came
    // from (itself where it bounced off a wall), so t_a = k_a (m(src_a) - r) +
    // dev_a, exact up to the rounding of that small sum.  Direction by
    // direction: one float4 load (four sets) per source node, the sets in
    // packed pairs, and the sums accumulated in the order a = 0..8, which every
    // evaluation of a node's fields shares.  rest(m4, p): the rest values of
    // pair p from a float4; dev(p, a): the pair's two deviations of direction
    // a; EDGE: the row may be the lattice's first or last (edge).
    template <int NPAIR, bool EDGE, class Dev, class Rest, class Acc>
    __device__ __forceinline__ static void diffs16(const char* base, const MomAddr& ma, const Edge& edge,
                                                   const Dev& dev, float4 m0, const Rest& rest,
                                                   const Acc& acc)
    {
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            float4 m4 = m0;
            switch (a) {   // (a is a constant once the loop is unrolled)
            case 1: m4 = mom_src<1, 0>(base, ma); break;
            case 2: m4 = mom_src<0, 1>(base, ma); break;
            case 3: m4 = mom_src<-1, 0>(base, ma); break;
            case 4: m4 = mom_src<0, -1>(base, ma); break;
            case 5: m4 = mom_src<1, 1>(base, ma); break;
            case 6: m4 = mom_src<-1, 1>(base, ma); break;
            case 7: m4 = mom_src<-1, -1>(base, ma); break;
            case 8: m4 = mom_src<1, -1>(base, ma); break;
            default: break;
            }
            if (EDGE) {
                const int ey = ey_dir(a), ex = ex_dir(a);
                if ((ey > 0 && edge.bounce_lo) || (ey < 0 && edge.bounce_hi)) m4 = m0;
                const float4* wrow = ey > 0 ? edge.wrap_lo : (ey < 0 ? edge.wrap_hi : nullptr);
                if (wrow) {
                    int x = edge.xg - ex;
                    x = x < 0 ? x + edge.nx : (x >= edge.nx ? x - edge.nx : x);
                    m4 = wrow[x];
                }
            }
#pragma unroll
            for (int p = 0; p < NPAIR; ++p)
                acc(p, a, fma2(f2(k_of_dir(a)), sub2(rest(m4, p), rest(m0, p)), dev(p, a)));
        }
    }
    template <bool EDGE, class Dev>
    __device__ __forceinline__ Mom rebuild_moments(const char* base, const MomAddr& ma, const Edge& edge,
                                                   const Dev& dev) const
    {
        const float4 m0 = *reinterpret_cast<const float4*>(base + ma.own);
        float2 dd[2], jx[2], jy[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) dd[p] = jx[p] = jy[p] = f2(0.0f);
        float gnd = 0.0f, gxy = 0.0f;
        diffs16<2, EDGE>(
            base, ma, edge,
            [&](int p, int a) { return s2f2<T16>(dev(9 * p + a)); },
            m0, [](const float4& v, int p) { return p == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w); },
            [&](int p, int a, float2 t) {
                const int ex = ex_dir(a), ey = ey_dir(a);
                dd[p] = add2(dd[p], t);
                if (ex > 0) jx[p] = add2(jx[p], t);
                if (ex < 0) jx[p] = sub2(jx[p], t);
                if (ey > 0) jy[p] = add2(jy[p], t);
                if (ey < 0) jy[p] = sub2(jy[p], t);
                if (p == 0) {
                    if (ex != 0 && ey == 0) gnd += t.y;
                    if (ex == 0 && ey != 0) gnd -= t.y;
                    if (ex != 0 && ey != 0) gxy += (ex * ey) * t.y;
                }
            });
        Mom m;
        m.f = SetMom{m0.x, dd[0].x, jx[0].x, jy[0].x};
        m.g = SetMom{m0.y, dd[0].y, jx[0].y, jy[0].y};
        m.h = SetMom{m0.z, dd[1].x, jx[1].x, jy[1].x};
        m.q = SetMom{m0.w, dd[1].y, jx[1].y, jy[1].y};
        m.gnd = gnd;
        m.gxy = gxy;
        return m;
    }
    __device__ __forceinline__ Mom own_moments(int st, int rb, int tx, int phys) const
    {
        const uint32_t* p = &sm.dev[st][0][rb][tx];
        const auto dev = [&](int i) { return p[i * TY * TX]; };
        const MomAddr ma = mom_addr(tx, rb);
        const char* base = mom_base(st);
        // a warp is one row: the edge test is uniform across it
        const bool edge = d.walls ? (phys == 1 || phys == d.ny - 2) : (phys == 0 || phys == d.ny - 1);
        if (edge) return rebuild_moments<true>(base, ma, edge_of(phys, tx), dev);
        return rebuild_moments<false>(base, ma, Edge{}, dev);
    }
    // The first 2 TY side threads take the second set pair (h, q) of the
    // inner columns, two columns per row; the other 4 TY the first pair of all
    // four side columns, four columns per row.  The threads of one warp then
    // read one set pair's planes (no two addresses in one shared-memory bank
    // within a 16-bit load), and each quarter warp the rest moments of four
    // columns (two rows per bank instead of eight).
    __device__ __forceinline__ static void side_slot(int it, int& item, int& rr)
    {
        if (it < 2 * TY) {
            rr = it >> 1;
            item = (it & 1) ? 5 : 3;     // inner column w or -1, pair (h, q)
            return;
        }
        const int a = it - 2 * TY;
        rr = a >> 2;
        const int col = a & 3;           // columns -2, -1, w, w + 1
        item = col == 0 ? 0 : (col == 1 ? 2 : (col == 2 ? 4 : 1));
    }
    // Side items: 0, 1: phi at the outer columns -2, w + 1; 2..5: the inner
    // columns -1, w, set pair (f, g) or (h, q).  Every item takes the same
    // two-set path (outer items use its first set), so that the lanes of a
    // warp do not split over set pairs; only the field update differs.
    template <int SL>
    __device__ __forceinline__ void side_item(int st, int item, int r, int phys, int rw,
                                              Window<SL>& W) const
    {
        const bool outer = item < 2;
        const int lr = outer ? item : (item - 2) / 2;
        const int f = outer ? 0 : (item - 2) % 2;
        const int c = outer ? (lr ? sp.w + 1 : -2) : (lr ? sp.w : -1);
        const int bc = lr ? c - sp.w : c + 8;
        const uint32_t* p = &sm.side[st][lr][9 * f][r][bc];
        constexpr int P = TY * 8;
        const MomAddr ma = mom_addr(c, r);
        const char* base = mom_base(st);
        const float4 m0 = *reinterpret_cast<const float4*>(base + ma.own);
        float2 dd = f2(0.0f);
        diffs16<1, true>(
            base, ma, edge_of(phys, c),
            [&](int, int a) { return s2f2<T16>(p[a * P]); }, m0,
            [f](const float4& v, int) { return f ? make_float2(v.z, v.w) : make_float2(v.x, v.y); },
            [&](int, int, float2 t) { dd = add2(dd, t); });
        const float d1 = dd.x, d2 = dd.y;
        const float s1 = fmaf(36.0f, f ? m0.z : m0.x, d1);
        if (outer) {
            put_side_phi(d, W, rw, phys, c, s1);
            return;
        }
        put_side_pair(d, W, rw, phys, c, f == 0 ? 1 : 2, s1, fmaf(36.0f, f ? m0.w : m0.y, d2));
    }
};

// ---- kernels --------------------------------------------------------------------------------

template <int S, int SLOTS, int BPS>
__global__ void __launch_bounds__(NT, BPS) stream32_kernel(const __grid_constant__ StreamBatchArgs args)
{
    extern __shared__ __align__(128) unsigned char s_raw[];
    auto& sm = *reinterpret_cast<Smem32<S, SLOTS>*>(s_raw);
    int s = 0;
    while (s + 1 < args.n && (int)blockIdx.x >= args.first[s + 1]) ++s;
    const LbmDev& d = args.dev[s];
    const Strip sp = strip_of(d, args.strip_chunks[s], blockIdx.x - args.first[s]);
    if (sp.c0 >= sp.c1) return;
    Stage32<S, SLOTS> stg{sm, d, sp, &args.tmap[s], &args.tside[s]};
    walk<S, SLOTS>(d, sp, stg, sm.win, sm.bar, args.err[s],
                   Out32{static_cast<float*>(args.dst[s]), d.nx * d.ny});
}

template <typename T16, int S, int SLOTS, int BPS>
__global__ void __launch_bounds__(NT, BPS) stream16_kernel(const __grid_constant__ Stream16Args args)
{
    extern __shared__ __align__(128) unsigned char s_raw[];
    auto& sm = *reinterpret_cast<Smem16<T16, S, SLOTS>*>(s_raw);
    int s = 0;
    while (s + 1 < args.n && (int)blockIdx.x >= args.first[s + 1]) ++s;
    const LbmDev& d = args.dev[s];
    const Strip sp = strip_of(d, args.strip_chunks[s], blockIdx.x - args.first[s]);
    if (sp.c0 >= sp.c1) return;
    Stage16<T16, S, SLOTS> stg{sm, d, sp, &args.tmap[s], &args.tside[s], &args.tmom[s],
                               static_cast<const float4*>(args.msrc[s])};
#if LBM_WALK_LAG
    walk_lag<S, SLOTS>(d, sp, stg, sm.win, sm.park, sm.bar, args.err[s],
                       Out16<T16>{static_cast<uint32_t*>(args.dst[s]),
                                  static_cast<float4*>(args.mdst[s]), d.nx * d.ny});
#else
    walk<S, SLOTS>(d, sp, stg, sm.win, sm.bar, args.err[s],
                   Out16<T16>{static_cast<uint32_t*>(args.dst[s]), static_cast<float4*>(args.mdst[s]),
                              d.nx * d.ny});
#endif
}

// Kernel configurations: one stage for either storage, refilled once the
// chunk's moments are taken (a second 16-bit stage measured 2 % slower: the
// kernel is issue-bound, and the stage's 35 KB come out of the L1 share);
// resident blocks per SM (kStreamBlocksPerSm).
constexpr int kS32 = 1, kSlots32 = kSlots, kBps32 = kStreamBlocksPerSm;
constexpr int kS16 = 1, kSlots16 = kSlots, kBps16 = kStreamBlocksPerSm;
constexpr int kSmem32 = (int)sizeof(Smem32<kS32, kSlots32>);
template <typename T16>
constexpr int smem16() { return (int)sizeof(Smem16<T16, kS16, kSlots16>); }

}  // namespace

inline cudaError_t prepare()
{
    cudaError_t e = cudaFuncSetAttribute(stream32_kernel<kS32, kSlots32, kBps32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem32);
#if LBM_STREAM_16BIT
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stream16_kernel<__half, kS16, kSlots16, kBps16>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem16<__half>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stream16_kernel<__nv_bfloat16, kS16, kSlots16, kBps16>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem16<__nv_bfloat16>());
#endif
    return e;
}

inline cudaError_t launch32(const StreamBatchArgs& args, cudaStream_t s)
{
    stream32_kernel<kS32, kSlots32, kBps32><<<args.first[args.n], dim3(TX, TY), kSmem32, s>>>(args);
    return cudaGetLastError();
}

inline cudaError_t launch16(const Stream16Args& args, int precision, cudaStream_t s)
{
#if LBM_STREAM_16BIT
    if (precision == LBM_FP16)
        stream16_kernel<__half, kS16, kSlots16, kBps16>
            <<<args.first[args.n], dim3(TX, TY), smem16<__half>(), s>>>(args);
    else if (precision == LBM_BF16)
        stream16_kernel<__nv_bfloat16, kS16, kSlots16, kBps16>
            <<<args.first[args.n], dim3(TX, TY), smem16<__nv_bfloat16>(), s>>>(args);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
#else
    (void)args, (void)precision, (void)s;
    return cudaErrorInvalidValue;   // no 16-bit kernels in this shape
#endif
}
