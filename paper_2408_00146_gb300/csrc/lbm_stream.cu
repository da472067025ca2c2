// lbm_stream.cu -- y-streaming step kernels (FP32 and 16-bit population
// storage) of the coupled central-moment LB system of arXiv 2408.00146.
//
// A block (256 threads) owns one column of the lattice, up to TX nodes wide,
// over a strip of chunks of TY rows and walks it in +y.  Two tile shapes are
// compiled, 32 x 8 and 64 x 4 (kStreamW, kStreamH; the second for FP32
// storage only), from one body (lbm_stream_body.cuh) included once per shape;
// the launch picks the shape that the batch's strip plan names.  Each chunk's populations (and,
// with 16-bit storage, the rest-state moments around it) arrive by TMA into
// a stage of shared memory.  The chunk's nodes are reduced right away to the
// few raw moments the collisions need (below), held in registers; the stage
// is then free for the next copy.  The macroscopic fields that the
// isotropic stencils read (phi, sigma(T, psi), p* - rho c_s^2, the normals)
// live in a circular window of rows in shared memory, indexed by physical
// row, so rows are never moved or loaded twice.  Rows beyond a wall are
// written as mirror images by the threads that compute the mirrored rows.
//
// Moment form of the collisions.  Every scheme relaxes the central moments
// of its populations (App. B-E), and all moments above first order of f, h
// and q, and all but the 2d and 11 moments of g, go to their equilibria with
// rate 1 (Eqs. (27), (33), (38), (43)).  The post-collision populations
// therefore depend on the pre-collision populations only through
//   f, h, q: the zeroth moment s and the first moments j (Eqs. (28), (39), (44));
//   g:       p*, j, sum g (e_x^2 - e_y^2) and sum g e_x e_y,
// fourteen numbers per node.  For f, h and q the post-collision central
// moments (s, a, b, s/3, s/3, 0, 0, 0, s/9) map back (P^-1 F(-u), App. F) to
//   v_ij = s E_i(u_x) E_j(u_y) + a O_i(u_x) Z_j(u_y) + b Z_i(u_x) O_j(u_y),
// with the one-dimensional populations E, Z, O of the moment triples
// (1, 0, 1/3), (1, 0, 0) and (0, 1, 0) about u.  The populations are formed as
// deviations from the weighted rest state, v = w s + dev, with
// dev = s (E E - w) + a O Z + b Z O, and w s = k m with the integer weights
// k = 36 w and m = s/36 (see Out32).  For g the nine post-collision central
// moments go through the factorised inverse transform.
#include "lbm_internal.h"
#include "lbm_device.cuh"

// LBM_WALK_LAG: the 16-bit kernels walk their strips with one barrier per
// chunk (walk_lag); the FP32 kernels keep two (walk), which measured 2.5 %
// faster for them.
namespace shape_32x8 {
constexpr int TX = 32, TY = 8;
#define LBM_STREAM_16BIT 1
#define LBM_WALK_LAG 1
#include "lbm_stream_body.cuh"
#undef LBM_WALK_LAG
#undef LBM_STREAM_16BIT
}  // namespace shape_32x8

// 64 x 4: FP32 storage only.  Its 16-bit kernel did not finish a step of the
// smallest case tried (one 64 x 160 lattice) and is not built.
namespace shape_64x4 {
constexpr int TX = 64, TY = 4;
#define LBM_STREAM_16BIT 0
#define LBM_WALK_LAG 0
#include "lbm_stream_body.cuh"
#undef LBM_WALK_LAG
#undef LBM_STREAM_16BIT
}  // namespace shape_64x4

static_assert(kStreamShapes == 2 && kStreamW[0] == shape_32x8::TX && kStreamH[0] == shape_32x8::TY &&
                  kStreamW[1] == shape_64x4::TX && kStreamH[1] == shape_64x4::TY,
              "shape table");

cudaError_t prepare_stream()
{
    cudaError_t e = shape_32x8::prepare();
    if (e == cudaSuccess) e = shape_64x4::prepare();
    return e;
}

bool stream_shape_available(int shape, int precision)
{
    return shape == 0 || precision == LBM_FP32;
}

bool stream_eligible(const LbmDev& d, int precision)
{
    const int align = precision == LBM_FP32 ? 4 : 8;
    if (d.nx % align != 0 || d.nx < 32 || d.nfy < 16) return false;
    if (d.walls) return true;
    // periodic y: whole chunks of every shape
    return d.nfy % 8 == 0;
}

int stream_columns(const LbmDev& d, int shape)
{
    return (d.nx + kStreamW[shape] - 1) / kStreamW[shape];
}

int stream_chunks(const LbmDev& d, int shape)
{
    return (d.nfy + kStreamH[shape] - 1) / kStreamH[shape];
}

int stream_blocks_per_sm(int) { return kStreamBlocksPerSm; }

int stream_blocks(const LbmDev& d, int strip_chunks, int shape)
{
    return stream_columns(d, shape) * ((stream_chunks(d, shape) + strip_chunks - 1) / strip_chunks);
}

cudaError_t launch_stream_batch(const StreamBatchArgs& args, int shape, cudaStream_t s)
{
    return shape == 0 ? shape_32x8::launch32(args, s) : shape_64x4::launch32(args, s);
}

cudaError_t launch_stream16_batch(const Stream16Args& args, int precision, int shape, cudaStream_t s)
{
    return shape == 0 ? shape_32x8::launch16(args, precision, s)
                      : shape_64x4::launch16(args, precision, s);
}
