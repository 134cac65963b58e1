// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (that is include/eles.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "eles.h"

namespace eles {

constexpr int kMaxRing = 64;      // largest ring (taps / stride + 1) of the strided-convolution tables
constexpr int kMaxStride = 8;     // largest DNS/LES stride of the banded ring kernels

// A banded operator A[nl][n]: row r has `T` entries starting at column
// start[r] (periodic operators wrap the column index modulo n).
struct Band {
    int n = 0, nl = 0, T = 0;
    int *d_start = nullptr;       // [nl]
    double *d_w64 = nullptr;      // [nl][T]
    float *d_w32 = nullptr;       // [nl][T]
};

// Strided convolution form of a periodic operator whose LES nodes coincide
// with DNS nodes (n = r nl): A[X][x] = w[x - r X] for |x - r X| <= R.
// Table W[s][dd] = w[s - r (dd + dmin)] for s in [0, r), dd in [0, D).
struct Ring {
    bool ok = false;
    int r = 0, R = 0, dmin = 0, dmax = 0, D = 0;
    double W64[kMaxStride * kMaxRing];
    float W32[kMaxStride * kMaxRing];
};

constexpr int kFusedMaxRows = 384;   // largest nz of the fused x-z kernel (one thread per z-row)

// Parameters of the fused x-z kernel (FP32).
struct FusedArgs {
    CUtensorMap tmap;     // TMA view of u: {nx, nz, 3 ny S} floats, box {8, box_rows, 1} (when use_tma)
    int use_tma, box_rows;
    const float *u;       // [S][3][ny][nz][nx]
    float *h;             // [S][9][ny][nlz][nlx]
    double *uref;         // [S][3][ny]
    double *plane_mean;   // [S][3][ny] or nullptr
    int nx, ny, nz, nlx, nlz;
    int nblk_x;           // x ring: blocks streamed per row (a multiple of the stage blocks)
    int bshift, dmin_x;   // stream block bi is row block bi - bshift (mod nlx); it completes X = bi - bshift + dmin
    int dmax_z, ZQs, NQ;  // z ring: dmax, Z outputs per work item, items per column
    int P, lP;            // completed columns parked per z phase (a power of two), log2 P
    int nf;               // fields to contract in z (9, or 3 for the velocities only)
    int *err;             // device error word
    float WX[kMaxStride * kMaxRing];
    float WZ[kMaxStride * kMaxRing];
};

// Tensor-core variant: FusedArgs plus the B fragments (hi and lo split) of
// the x-operator tile, two 32-bit words per lane.
struct FusedTCArgs {
    FusedArgs f;
    unsigned Bh[64];
    unsigned Bl[64];
    int KS = 0, zoff = 0;          // tensor-core z phase: k-steps per Z tile, window offset (KS 0: CUDA cores)
    const uint4 *afrag = nullptr;  // its A fragments [KS][32][hi, lo] (device)
};
bool tc_supported(int rx, int dx, int rz, int dz, int nlz);
void tc_weights(const Ring &rx, FusedTCArgs *ta);
size_t tc_smem_bytes(int P, int nz, int KS);
// Encode the TMA view of a batch of snapshots u [S][3][ny][nz][nx] (host).
int encode_u_map(const float *u, int nx, int ny, int nz, int nsnap, int box_w, int box_rows, CUtensorMap *map);
cudaError_t launch_fused_tc(int rz, int dz, const FusedTCArgs &ta, int nsnap, cudaStream_t st);
int tc_zfrags(const Ring &rz, int nlz, std::vector<unsigned> &out, int *zoff_out);

// Warp-specialised tensor-core x-z kernel (xz_ws.cuh, x_variant 3) for the
// split-precision plans: the grid heights it is instantiated for, and its
// per-plan tables.
#define ELES_WS_NZ_LIST(X) X(64) X(128) X(192) X(256) X(384)
struct WsHost {
    bool ok = false;
    int mode = 0;                 // ws::MODE_BF16X3 or ws::MODE_TF32X2
    int OP = 1, OPC = 2, CB = 2;  // output phases, outputs per chunk and phase, x blocks per chunk
    int bshift = 0, nchunk = 0;   // x stream
    int xc0[4] = {0, 0, 0, 0};    // first output completed by chunk 0, per phase
    int KS = 0, zoff = 0;         // tensor-core z phase
    unsigned *d_afrag = nullptr;  // z A fragments (device)
    unsigned *d_bvar = nullptr;   // rotated x B fragments (device)
};

bool fused_supported(int rx, int dx, int rz, int dz);
int fused_stage_blocks(int rx);
size_t fused_smem_bytes(int rx, int P, int nz);
cudaError_t launch_fused(int rx, int dx, int rz, int dz, const FusedArgs &a, int nsnap, cudaStream_t st);

// Parameters of the y-contraction and recovery (any precision).
template <typename T>
struct YArgs {
    const T *h;            // [S][9][ny][nlz][nlx]
    const T *wy;           // [S][nly][ny][8]: w+, w-, U1 w+, U1 w-, U2 w+, U2 w-, U3 w+, U3 w-
    const double *AU;      // [S][3][nly]
    const double *AUU;     // [S][6][nly]
    const int *ystart, *ycount;
    T *ubar, *tau;         // [S][3][..], [S][6][..]
    T *tmp;                // [S][12][nly][nlz][nlx]: q_a and C_ab between the two passes
    int ny, nly, nlz, nlx;
    int stress, flip;      // flip: Eq. 9 parities
    int ptrans;            // h planes in (X, Z) order; outputs are written in (Z, X) order
    int *err;
};

// Tensor-core y passes for EF_PREC_BF16X3 (ypass_tc.cu): the banded y
// operators as split-BF16 A fragments per 16-row LES tile and 16-row k-step,
// h of a field triple staged in shared memory by TMA.
constexpr int kYMaxTiles = 32;     // LES row tiles of 16 (nly <= 512)
constexpr int kYOps = 9;           // y operators per snapshot (A+, A-, A- - A+, six deviation-folded)
constexpr int kYTmp = 21;          // scratch slots: q_a, C'_ab, d_a, q_11 .. q_33
struct YTcGeom {
    int nmt = 0;                   // LES row tiles
    int jb[kYMaxTiles] = {};       // first DNS row of tile mt's band
    int ks[kYMaxTiles] = {};       // its 16-row k-steps
    int koff[kYMaxTiles] = {};     // their offset in the fragment table
    int kstot = 0;                 // k-steps of all tiles
    int box_rows = 0;              // TMA box rows (two boxes stage the band rows of every tile)
    int dzero[kYMaxTiles] = {};    // 1: A_y^- = A_y^+ on every row of tile mt (its wall term d is zero)
};
struct YTcArgs {
    CUtensorMap hmap;              // TMA view of h: {nplane, 9 ny S} floats, box {36, box_rows}
    YTcGeom geo;
    const uint4 *frag;             // [S][kYOps][kstot][hi, lo][32 lanes]
    const double *AU;              // [S][3][nly]
    const float *Kab;              // [S][6][nly]: A_y(U_a U_b) - A_y U_a A_y U_b
    float *ubar, *tau;             // [S][3][nly][nplane], [S][6][nly][nplane]
    float *tmp;                    // [S][kYTmp][nly][nplane]
    int ny, nly, nplane, stress, flip;
    int nlz, nlx, ptrans;          // ptrans: h planes in (X, Z) order; outputs are written in (Z, X) order
    int nsnap;                     // snapshots of the launch (range checks)
    int *err;
};
bool ytc_geometry(const std::vector<int> &ystart, const std::vector<int> &ycount, int ny, int nplane, YTcGeom *g);
cudaError_t launch_yfrag(const YTcGeom &g, const double *yw_even, const double *yw_odd, const double *uref,
                         const double *AU, int ny, int nly, int nsnap, uint4 *frag, cudaStream_t st);
int encode_h_map(const float *h, int nplane, int ny, int nsnap, int box_rows, CUtensorMap *map);
cudaError_t launch_ytc(const YTcArgs &a, int nsnap, cudaStream_t st);

template <typename T>
cudaError_t launch_yprofile(const double *uref, const int *ystart, const int *ycount, const double *we,
                            const double *wo, int ny, int nly, int flip, int nsnap, double *AU, double *AUU,
                            T *wy, float *Kab, cudaStream_t st);
template <typename T>
cudaError_t launch_ypass(const YArgs<T> &a, int nsnap, cudaStream_t st);

}  // namespace eles

namespace eles { struct DiffPlan; }

// NVTX range over a host-side scope (visible to profilers; free otherwise).
#include <nvtx3/nvToolsExt.h>
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct ef_plan {
    int device = 0;
    int nx = 0, ny = 0, nz = 0, nlx = 0, nly = 0, nlz = 0;
    double Lx = 0, Lz = 0, delta = 0;
    int ext = 0, prec = 0;
    int yquad = 0;                // y quadrature: 0 trapezoid, 1 hat (EF_KERNEL_GAUSSIAN_HAT)
    eles::DiffPlan *diff = nullptr;   // EF_KERNEL_DIFFERENTIAL: its transforms and scratch
    int par[3] = {1, -1, 1};      // wall parity of u1, u2, u3 (Eq. 7 or Eq. 9)
    eles::Band bx, bz;            // x and z operators
    eles::Ring rx, rz;            // their strided-convolution tables (if ok)
    int x_variant = 0;            // 0 generic gather, 1 ring (CUDA cores), 2 tensor cores,
                                  // 3 tensor cores, warp-specialised
    // y operators, dense [nly][ny] rows with a nonzero range per row
    int *d_ystart = nullptr, *d_ycount = nullptr;
    double *d_yw64[2] = {nullptr, nullptr};   // [0] even, [1] odd
    float *d_yw32[2] = {nullptr, nullptr};
    int ytaps_max = 0;
    bool ytc_ok = false;          // tensor-core y passes (EF_PREC_BF16X3)
    bool ytc_fit = false;         // the banded y tiling fits this geometry (ytc_ok unless switched off)
    unsigned gen = 0;             // bumped whenever scratch or the kernel choice changes (batch graphs re-capture)
    long long wait_limit = 0;     // bound of one device wait in SM clocks (0: the default, about 2 s)
    eles::YTcGeom ytc;            // their banded tiling
    uint4 *d_yfrag = nullptr;     // their A fragments, [S][kYOps][kstot][2][32]
    double *d_ygrid = nullptr;    // DNS y nodes on the device
    bool fused = false;           // FP32 fused x-z kernel available for this plan
    int NQ = 1, ZQs = 0, P = 8;   // its z work split and columns per z phase
    int bshift = 0, nblk_x = 0;   // its x stream
    eles::FusedTCArgs tc;         // tensor-core B fragments (x_variant 2)
    bool tc_ok = false;           // the tensor-core x-z kernel supports this plan
    eles::WsHost ws;              // the warp-specialised tensor-core kernel (x_variant 3), if ok
    uint4 *d_zfrag = nullptr;     // tensor-core z-phase A fragments (x_variant 2)
    // scratch owned by the plan, sized for `reserve` snapshots per launch
    int reserve = 0;
    void *d_g = nullptr;          // x-contracted fields of one snapshot [9][ny][nz][nlx] (unfused path)
    void *d_h = nullptr;          // x,z-contracted fields [S][9][ny][nlz][nlx]
    double *d_uref = nullptr;     // reference profile U_c(y_j), [S][3][ny]
    void *d_urefT = nullptr;      // same in the working type, one snapshot
    double *d_rowsum = nullptr;   // partial sums of the fluctuation, [3][ny][nzw], one snapshot
    int nzw = 0;
    double *d_AU = nullptr;       // A_y U_c, [S][3][nly]
    double *d_AUU = nullptr;      // A_y (U_a U_b), [S][6][nly]
    float *d_Kab = nullptr;       // A_y (U_a U_b) - A_y U_a A_y U_b, [S][6][nly]
    void *d_wy = nullptr;         // y weights with U folded in, [S][nly][ny][8]
    void *d_ytmp = nullptr;       // partial sums between the y passes, [S][kYTmp][nly][nlz][nlx]
    int *d_err = nullptr;         // device error word
    // phase timing (ef_profile_enable)
    bool prof_on = false;
    static constexpr int kProfSlots = 64, kProfEvents = 5;
    cudaEvent_t prof_ev[kProfSlots][kProfEvents] = {};
    bool prof_used[kProfSlots] = {};
    long prof_calls = 0;
    double prof_ms[4] = {0, 0, 0, 0};
};

namespace eles {

// Every device allocation of the library goes through these, so that a test
// hook (ef_debug_fail_alloc) can make the n-th next one fail.
cudaError_t dev_malloc_void(void **p, size_t bytes);
cudaError_t dev_malloc_async_void(void **p, size_t bytes, cudaStream_t s);
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes) { return dev_malloc_void(reinterpret_cast<void **>(p), bytes); }
template <typename T>
inline cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t s)
{
    return dev_malloc_async_void(reinterpret_cast<void **>(p), bytes, s);
}

// Range checks of global indices in the debug build (-DELES_CHECK): a
// violation records EF_ERR_RANGE in the error word and the access is skipped;
// nothing traps.  In the normal build the check is the constant true.
#ifdef ELES_CHECK
__device__ __forceinline__ bool in_range(size_t i, size_t n, int *err)
{
    if (i < n) return true;
    if (err) atomicCAS(err, 0, (int)EF_ERR_RANGE);
    return false;
}
#else
__device__ __forceinline__ constexpr bool in_range(size_t, size_t, int *) { return true; }
#endif

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// setup_kernels.cu
int build_periodic_band(int n, double L, int nl, double delta, Band *b);
int build_ring(const Band &b, Ring *r);
int build_wall_rows(ef_plan *p, const double *h_les_y);

// Phase events of the current call (nullptr entries when timing is off).
struct PhaseEvents { cudaEvent_t e[ef_plan::kProfEvents]; };
int prof_begin(ef_plan *p, PhaseEvents *pe);
inline void prof_mark(const PhaseEvents *pe, int k, cudaStream_t s)
{
    if (pe && pe->e[k]) cudaEventRecord(pe->e[k], s);
}

// filter_kernels.cu
int run_filter(ef_plan *p, int nsnap, const void *u, void *ubar, void *tau, double *plane_mean,
               bool stress, cudaStream_t s, const PhaseEvents *pe);
int plan_reserve(ef_plan *p, int nsnap);

// xz_ws.cu
int ws_setup(ef_plan *p, const char **why);
void ws_free(WsHost &w);
int ws_run(const ef_plan *p, int nsnap, const float *u, float *h, double *uref, double *plane_mean, int nf,
           cudaStream_t st);
int ws_run_batch(ef_plan *const *plans, const int *nsnap, const float *const *u, int n, int nf, cudaStream_t st);
// filter_kernels.cu: the y stage of a plan whose h (and profile) are in place
int run_y_stage(ef_plan *p, int nsnap, void *ubar, void *tau, bool stress, cudaStream_t s);

// closure_tc.cu: tensor-core inference of the closure MLP.  `image` is a
// device buffer of closure_tc_image_bytes() that the call repacks from the
// working weights and statistics; nfall counts guarded points; err receives
// EF_ERR_TIMEOUT if a wait ran out.
// differential.cu: the differential filter (EF_KERNEL_DIFFERENTIAL, FP64)
int diff_setup(ef_plan *p, const double *dns_y, const double *les_y);
void diff_destroy(DiffPlan *d);
int diff_run(ef_plan *p, int nsnap, const void *u, void *ubar, void *tau, double *plane_mean, bool stress,
             cudaStream_t s);

size_t closure_tc_image_bytes();
// The exact-stress fallback of the closure through a filter plan (closure_tc.cu).
struct ExactFallbackArgs {
    const float *feats;          // [n][10]
    long n;
    float guard;
    const unsigned char *image;  // the packed inference image (its statistics)
    const float *u32;            // DNS snapshot [3][ny][nz][nx] (FP32 plans) ...
    const double *u64;           // ... or FP64 (FP64 plans); the other is NULL
    size_t np;                   // nx ny nz
    int nx, ny, nz, nlx, nly, nlz;
    const int *xstart, *zstart;  // the banded x and z operators [nl][T]
    const double *xw, *zw;
    int Tx, Tz;
    const int *ystart, *ycount;  // the y operators, dense [nly][ny] per parity (even, odd)
    const double *yw[2];
    int par[3];                  // wall parities of u1, u2, u3
    float *tau;                  // [6][n]: overwritten at the guarded points
};
int closure_exact_fallback(const ExactFallbackArgs &a, cudaStream_t s);
int closure_infer_tc(const float *wq, const long *off_w, const long *off_b, const double *stats, void *image,
                     const float *feats, long n, float guard, const float *exact, float *tau, int *nfall, int *err,
                     cudaStream_t s);

}  // namespace eles
