// lbm_internal.h -- device-side parameter block and launch wrappers shared by
// the C-ABI layer (lbm_api.cu) and the kernels (lbm_kernels.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

// Records msg as the calling thread's lbm_last_error() text and returns st.
__attribute__((visibility("hidden"))) lbm_status lbm_set_error(lbm_status st, const char* msg);

// Lattice parameters in the form the kernels use them (FP32), derived on the
// host from lbm_params (Sec. 2, Sec. 6, App. B-E).
struct LbmDev {
    int nx, ny, walls;
    int y0;    // first fluid row (1 with walls, 0 without)
    int nfy;   // number of fluid rows
    // phase field (App. B): kappa_eq,10 = M_phi theta n_x, theta = 4 phi(1-phi)/W
    float W, mphi_4_over_W, omega_phi;
    // surfactant (App. E): rate, adsorption-flux coefficient m_psi and the
    // derivative of the Eq. (5) bracket G'(phi) = (phi - 1/2)(c_s32 phi(1-phi) + w)
    float omega_psi, m_psi, g_s32, g_w;
    // property interpolation, Eq. (17) (phi_A = 0, phi_B = 1)
    float rhoA, drho, muA, dmu, alphaA, dalpha;
    // surface tension law, Eq. (6)
    float sigma0, s0beta_over_Tref, sigma_T, sigma_TT, T_ref;
    float T_H, T_C;
    // CSF: delta_s = 1.5 W |grad phi|^2 (Sec. 3)
    float deltas_coef;
    float Fext_x, Fext_y, gravity;
    // analytic initial state
    float R, xb, yb, psi0;
    // surfactant at the walls: psi_bc 0 zero flux, 1 held at psi_L (y=0) and
    // psi_R (y=ny-1), 2 zero flux with the psi_L -> psi_R initial profile
    float psi_L, psi_R;
    int psi_bc;
};

// Tile shape of the fused step kernel.
constexpr int kTileX = 32;
constexpr int kTileY = 8;

// tmap: TMA descriptor of the population tensor [36][ny][nx] at src (box
// {kTileX, kTileY, 36}), or NULL to stage every tile with per-thread loads.
// err: device flag set to 1 if a bounded wait for a tile copy gave up.
cudaError_t launch_step(const LbmDev& d, const float* src, float* dst, const CUtensorMap* tmap,
                        int* err, cudaStream_t s);
cudaError_t launch_fields(const LbmDev& d, const float* src, float* fields, const CUtensorMap* tmap,
                          int* err, cudaStream_t s);
// One launch stepping up to kMaxBatch simulations (lbm_step_batch): the grid
// is the concatenation of every simulation's tiles; first[] holds the prefix
// sums of the tile counts.  Passed by value as a kernel parameter.
constexpr int kMaxBatch = 64;
struct BatchArgs {
    CUtensorMap tmap[kMaxBatch];  // 64-byte aligned descriptors (first member)
    LbmDev dev[kMaxBatch];
    const void* src[kMaxBatch];   // populations (FP32) or deviations (16-bit)
    void* dst[kMaxBatch];
    const void* msrc[kMaxBatch];  // rest-state moments (float4 per node), 16-bit storage only
    void* mdst[kMaxBatch];
    int* err[kMaxBatch];
    int first[kMaxBatch + 1];
    int has_tmap[kMaxBatch];
    int n;
};
cudaError_t launch_step_batch(const BatchArgs& args, int total_tiles, cudaStream_t s);
int tiles_of(const LbmDev& d);

// 16-bit population storage (precision LBM_FP16 / LBM_BF16): deviations
// dev[36][ny][nx] from the rest states mom[ny][nx] (float4: f, g, h, q).
// prepare_dev_storage: per-device kernel attributes, before the first launch.
cudaError_t prepare_dev_storage(int precision);
// One step dsrc/msrc -> ddst/mdst, or, with fields != NULL, the fields of the
// state dsrc/msrc ([6][ny][nx], as launch_fields).
cudaError_t launch_step_dev(const LbmDev& d, int precision, const void* dsrc, const float4* msrc,
                            void* ddst, float4* mdst, float* fields, cudaStream_t s);
// Batched step of sims that all have this precision (src/dst/msrc/mdst used).
cudaError_t launch_step_batch_dev(const BatchArgs& args, int precision, int total_tiles,
                                  cudaStream_t s);
// Initial state from the fields (as launch_init_equilibrium).
cudaError_t launch_init_dev(const LbmDev& d, int precision, const float* fields, void* dev,
                            float4* mom, cudaStream_t s);
// FP32 population planes a0 .. a0+count-1 (planes[count][ny][nx]) to
// deviations from mom, and back (join writes 0 on wall rows).  split sums
// the deviations' rounding errors per node and set into lost (a float4 per
// node, cleared when a0 == 0); launch_fold_lost then adds them to mom.
cudaError_t launch_split_planes(const LbmDev& d, int precision, const float* planes, int a0,
                                int count, const float4* mom, void* dev, float4* lost,
                                cudaStream_t s);
cudaError_t launch_fold_lost(const LbmDev& d, float4* mom, const float4* lost, cudaStream_t s);
cudaError_t launch_join_planes(const LbmDev& d, int precision, const void* dev, const float4* mom,
                               int a0, int count, float* planes, cudaStream_t s);

// Streaming steps of up to kMaxBatch (FP32) or kMaxBatch16 (16-bit storage)
// simulations per launch, in one of kStreamShapes tile shapes: blocks of
// 256 threads walk columns of up to kStreamW[shape] nodes in +y over strips
// of strip_chunks[s] chunks of kStreamH[shape] rows, reading the populations
// through TMA descriptors of the source buffer made for that shape: tmap[s]
// (box {W, H, 36}) and tside[s] (side columns: box {4, H, 36} for FP32,
// {8, H, 36} for 16-bit deviations), and, with 16-bit storage, tmom[s]
// (rest-state moments, the float4 array viewed as [ny][nx][4] floats, box
// {4, 8, H + 2}); first[] holds the prefix sums of stream_blocks.
// prepare_stream: per-device kernel attributes, before the first launch.
constexpr int kStreamShapes = 2;
constexpr int kStreamW[kStreamShapes] = {32, 64};
constexpr int kStreamH[kStreamShapes] = {8, 4};
constexpr int kStreamBlocksPerSm = 2;
struct StreamBatchArgs {
    CUtensorMap tmap[kMaxBatch];
    CUtensorMap tside[kMaxBatch];
    LbmDev dev[kMaxBatch];
    void* dst[kMaxBatch];
    int* err[kMaxBatch];
    int strip_chunks[kMaxBatch];
    int first[kMaxBatch + 1];
    int n;
};
constexpr int kMaxBatch16 = 48;
struct Stream16Args {
    CUtensorMap tmap[kMaxBatch16];
    CUtensorMap tside[kMaxBatch16];
    CUtensorMap tmom[kMaxBatch16];
    LbmDev dev[kMaxBatch16];
    void* dst[kMaxBatch16];     // deviations of the destination buffer
    void* mdst[kMaxBatch16];    // rest-state moments of the destination buffer
    const void* msrc[kMaxBatch16];  // and of the source buffer (periodic y: wrapped rows)
    int* err[kMaxBatch16];
    int strip_chunks[kMaxBatch16];
    int first[kMaxBatch16 + 1];
    int n;
};
static_assert(sizeof(StreamBatchArgs) <= 32764 && sizeof(Stream16Args) <= 32764,
              "kernel parameter limit");
cudaError_t prepare_stream();
// Whether a lattice of this storage precision can be stepped by the
// streaming kernels: nx >= 32 and a multiple of 4 (FP32) or 8 (16-bit:
// 16-byte TMA rows), at least 16 fluid rows, and walls or a periodic y axis
// of whole 8-row chunks.  The same lattices for every shape.
bool stream_eligible(const LbmDev& d, int precision);
// Whether the tile shape has kernels for this storage precision (64 x 4:
// FP32 only).
bool stream_shape_available(int shape, int precision);
int stream_columns(const LbmDev& d, int shape);
int stream_chunks(const LbmDev& d, int shape);
// Resident blocks per SM of the streaming kernels.
int stream_blocks_per_sm(int precision);
int stream_blocks(const LbmDev& d, int strip_chunks, int shape);
cudaError_t launch_stream_batch(const StreamBatchArgs& args, int shape, cudaStream_t s);
cudaError_t launch_stream16_batch(const Stream16Args& args, int precision, int shape, cudaStream_t s);

// Diagnostic: one block waits with the kernels' bounded wait (limit_ns) on a
// barrier nothing completes and sets *flag = 1 when it gives up.
cudaError_t launch_bounded_wait_probe(uint64_t limit_ns, int* flag, cudaStream_t s);

cudaError_t launch_analytic_fields(const LbmDev& d, float* fields, cudaStream_t s);
cudaError_t launch_init_equilibrium(const LbmDev& d, const float* fields, float* pops,
                                    cudaStream_t s);
// FP64 reduction of the observables over fluid nodes into result[0..7]:
// sum phi, sum psi, sum phi x, sum phi y, sum phi u_x, sum phi u_y,
// non-finite count, fluid node count.  partials holds nblocks * 8 doubles.
cudaError_t launch_observe_reduce(const LbmDev& d, const float* fields, double* partials,
                                  int nblocks, double* result, cudaStream_t s);
constexpr int kReduceBlocks = 304;  // 2 x 152 SMs
constexpr int kReduceThreads = 256;
