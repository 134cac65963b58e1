// Host side of the warp-specialised tensor-core x-z kernel (xz_ws.cuh): the
// choice of output phases, the rotated x-operator B fragments of both split
// forms, the z-operator A fragments, and the launch.  This file instantiates
// the BF16X3 kernels; xz_ws_tf32.cu the TF32X2 ones.
#include <math.h>
#include <string.h>

#include <vector>

#include "eles_internal.h"
#include "xz_ws.cuh"

namespace eles {

namespace {

unsigned short bf16_bits(double w)
{
    const float x = (float)w;
    unsigned u;
    memcpy(&u, &x, 4);
    return (unsigned short)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}
double bf16_value(unsigned short b)
{
    const unsigned u = (unsigned)b << 16;
    float x;
    memcpy(&x, &u, 4);
    return x;
}
// TF32 (10 explicit mantissa bits) nearest to w, ties away from zero, as
// FP32 bits with the 13 low bits clear.
unsigned tf32_bits(double w)
{
    const float x = (float)w;
    unsigned u;
    memcpy(&u, &x, 4);
    return (u + 0x1000u) & 0xffffe000u;
}
double tf32_value(unsigned b)
{
    float x;
    memcpy(&x, &b, 4);
    return x;
}
// IEEE binary16 nearest to w (ties to even), for |w| < 65504.
unsigned short f16_bits(double w)
{
    if (w == 0.0) return 0;
    const unsigned short sign = w < 0 ? 0x8000u : 0u;
    const double a = fabs(w);
    int e = 0;
    const double m = frexp(a, &e);                 // a = m 2^e, m in [0.5, 1)
    const int E = e - 1 + 15;                      // biased exponent of a = 2m 2^(e-1)
    if (E <= 0) {                                  // subnormal: multiples of 2^-24
        const double r = nearbyint(ldexp(a, 24));  // 1024 rounds up to the smallest normal
        return (unsigned short)(sign | (unsigned)r);
    }
    double f = nearbyint((2.0 * m - 1.0) * 1024.0);
    unsigned bits = (unsigned)E << 10;
    if (f >= 1024.0) { bits = (unsigned)(E + 1) << 10; f = 0.0; }
    return (unsigned short)(sign | bits | (unsigned)f);
}
double f16_value(unsigned short b)
{
    const int E = (b >> 10) & 31, f = b & 1023;
    const double v = E ? ldexp(1.0 + f / 1024.0, E - 15) : ldexp((double)f, -24);
    return (b & 0x8000u) ? -v : v;
}

// Weight of chunk input xi (0..15) to phase output n (0..6) of a stream
// whose chunk 0 completes output xc0 first; n = 7 is the row-sum column.
double bweight(const Ring &r, int xi, int n, int xc0, int OP, int bshift)
{
    if (n == 7) return 1.0;
    const int dd = xc0 + OP * n + bshift - xi / r.r - r.dmin;
    return (dd >= 0 && dd < r.D) ? r.W64[(xi % r.r) * r.D + dd] : 0.0;
}

// Reference profile U_c(y_j): the mean of z-row 0 of each plane, one warp
// per (component, plane, snapshot).  Any profile makes the decomposition
// exact; this one is stored rounded to FP32, and the kernel and the recovery
// both use the stored value.  Each lane sums its 16-byte pieces of the row in
// FP32 (four for nx = 512), the lanes' sums are added in FP64.
__global__ void __launch_bounds__(96) ws_uref(const float *__restrict__ u, int nx, int ny, int nz, double *uref,
                                               int *err)
{
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31, j = blockIdx.x, s = blockIdx.y;
    const size_t r0 = (((size_t)s * 3 + c) * ny + j) * (size_t)nz * nx;
    const size_t nu = (size_t)gridDim.y * 3 * ny * nz * nx;
    double acc = 0.0;
    if ((nx & 3) == 0) {   // rows start on 16-byte boundaries (u is 16-byte aligned for TMA)
        const float4 *q = reinterpret_cast<const float4 *>(u + r0);
        float part = 0.f;
#pragma unroll 4
        for (int i = lane; i < nx / 4; i += 32)
            if (in_range(r0 + 4 * (size_t)i + 3, nu, err)) {
                const float4 v = __ldg(q + i);
                part += (v.x + v.y) + (v.z + v.w);
            }
        acc = part;
    } else {
        for (int i = lane; i < nx; i += 32)
            if (in_range(r0 + i, nu, err)) acc += (double)u[r0 + i];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const size_t k = ((size_t)s * 3 + c) * ny + j;
    if (lane == 0 && in_range(k, (size_t)gridDim.y * 3 * ny, err)) uref[k] = (double)(float)(acc / nx);
}

}  // namespace

// z-operator A fragments for the tensor-core z phase: k-step kk, lane
// (g, t) holds A[g][2t..2t+1], A[g+8][2t..2t+1], A[g][2t+8..2t+9],
// A[g+8][2t+8..2t+9] with A[m][k] = w[16 kk + r(k) - RZ m - zoff], split into
// hi and lo pairs twice: bf16 (for the velocity columns) and FP16 (for the
// product columns); r(2i + e) = i + 8e is the row order of the parked pairs.
// Layout [KS][bf16 hi, bf16 lo, f16 hi, f16 lo][32 lanes] uint4.  Returns
// KS (0 if the z operator does not qualify).
int ws_zfrags(const Ring &rz, int nlz, std::vector<unsigned> &out, int *zoff_out)
{
    if (!rz.ok || nlz % 16 != 0) return 0;
    const int R = rz.R, RZ = rz.r;
    const int zoff = (R + 15) / 16 * 16;   // window starts on 16-row boundaries
    const int KS = (zoff + 15 * RZ + R + 1 + 15) / 16;
    auto w = [&](int o) -> double {        // weight at offset o = z - RZ Z
        if (o < -R || o > R) return 0.0;
        const int e = ((o % RZ) + RZ) % RZ;
        const int dd = (e - o) / RZ - rz.dmin;
        return (dd >= 0 && dd < rz.D) ? rz.W64[e * rz.D + dd] : 0.0;
    };
    out.assign((size_t)KS * 4 * 32 * 4, 0u);
    for (int kk = 0; kk < KS; kk++)
        for (int lane = 0; lane < 32; lane++) {
            const int g = lane / 4, t = lane % 4;
            const int rows[4] = {g, g + 8, g, g + 8}, kofs[4] = {0, 0, 8, 8};
            for (int r = 0; r < 4; r++) {
                unsigned bh = 0, bl = 0, fh = 0, fl = 0;
                for (int e = 0; e < 2; e++) {
                    const int k = 2 * t + kofs[r] + e;
                    const int row = (k >> 1) + 8 * (k & 1);
                    const double v = w(16 * kk + row - RZ * rows[r] - zoff);
                    const unsigned short h = bf16_bits(v), l = bf16_bits(v - bf16_value(h));
                    const unsigned short h16 = f16_bits(v), l16 = f16_bits(v - f16_value(h16));
                    bh |= (unsigned)h << (16 * e);
                    bl |= (unsigned)l << (16 * e);
                    fh |= (unsigned)h16 << (16 * e);
                    fl |= (unsigned)l16 << (16 * e);
                }
                const unsigned words[4] = {bh, bl, fh, fl};
                for (int wd = 0; wd < 4; wd++) out[((size_t)(4 * kk + wd) * 32 + lane) * 4 + r] = words[wd];
            }
        }
    *zoff_out = zoff;
    return KS;
}

size_t ws_smem(int nz, int mode, int opc, int KS)
{
    using namespace ws;
#define ELES_WS_SMEM(NZ)                                                                                  \
    if (nz == NZ) {                                                                                       \
        if (mode == MODE_BF16X3) return opc == 2 ? ws_smem_bytes<NZ, MODE_BF16X3, 2>(KS)                 \
                                                 : ws_smem_bytes<NZ, MODE_BF16X3, 1>(KS);                 \
        return opc == 2 ? ws_smem_bytes<NZ, MODE_TF32X2, 2>(KS) : ws_smem_bytes<NZ, MODE_TF32X2, 1>(KS);  \
    }
    ELES_WS_NZ_LIST(ELES_WS_SMEM)
#undef ELES_WS_SMEM
    return 0;
}

bool ws_nz_supported(int nz)
{
#define ELES_WS_HAS(NZ) if (nz == NZ) return true;
    ELES_WS_NZ_LIST(ELES_WS_HAS)
#undef ELES_WS_HAS
    return false;
}

// Plan the kernel for a split-precision plan: output phases, B and z
// fragments (uploaded to the device).  Leaves p->ws.ok false (and says why in
// *why) when the grid or filter does not fit the kernel.
int ws_setup(ef_plan *p, const char **why)
{
    WsHost &w = p->ws;
    w = WsHost();
    *why = nullptr;
    const int mode = p->prec == EF_PREC_TF32X2 ? ws::MODE_TF32X2 : ws::MODE_BF16X3;
    const Ring &rx = p->rx, &rz = p->rz;
    if (!rx.ok || !rz.ok) { *why = "the LES x and z nodes must be every r-th DNS node"; return EF_OK; }
    if (rx.r != 4 && rx.r != 8 && rx.r != 16) { *why = "the x stride must be 4, 8 or 16"; return EF_OK; }
    if (!ws_nz_supported(p->nz)) { *why = "nz must be 64, 128, 192, 256 or 384"; return EF_OK; }
    if (p->nlz % 16 != 0) { *why = "the LES nz must be a multiple of 16"; return EF_OK; }
    const int CB = 16 / rx.r;
    if (p->nlx % CB != 0) { *why = "the LES nx must be a multiple of 16 / (x stride)"; return EF_OK; }
    const int bshift = (rx.dmax + CB - 1) / CB * CB;
    // output phases: the fewest whose window (plus the idle row-sum column)
    // fits 8 tile columns in every phase
    int OP = 0;
    int xc0[4] = {0, 0, 0, 0};
    for (int op = 1; op <= 4 && !OP; op *= 2) {
        if (CB % op != 0 || CB / op > 2) continue;
        bool fits = true;
        for (int ph = 0; ph < op; ph++) {
            const int first = rx.dmin - bshift;               // outputs completed by chunk 0: [first, first + CB)
            const int x0 = first + (((ph - first) % op) + op) % op;
            xc0[ph] = x0;
            const int delta = x0 + bshift - rx.dmin;          // in [0, op)
            if (delta + 7 * op - (CB - 1) < rx.D) fits = false;
        }
        if (fits) OP = op;
    }
    if (!OP) { *why = "the x filter is too wide for the tensor-core window (ring depth)"; return EF_OK; }
    const int OPC = CB / OP, NR = 8 / OPC;
    std::vector<unsigned> zf;
    int zoff = 0;
    const int KS = ws_zfrags(rz, p->nlz, zf, &zoff);
    if (KS <= 0 || 2 * zoff > p->nz) { *why = "the z filter is too wide for the tensor-core z phase"; return EF_OK; }
    if (ws_smem(p->nz, mode, OPC, KS) > 227 * 1024 - 256) {   // static shared memory included
        *why = "the kernel's shared memory exceeds 227 KB for this grid";
        return EF_OK;
    }
    // rotated B fragments per phase: [OP][NR][32][BW] uint4, the velocities'
    // words first, the products' FP16 words last
    const int BW = mode == ws::MODE_TF32X2 ? 3 : 2;
    std::vector<unsigned> bv((size_t)OP * NR * 32 * BW * 4, 0u);
    for (int ph = 0; ph < OP; ph++)
        for (int q = 0; q < NR; q++)
            for (int lane = 0; lane < 32; lane++) {
                const int g = lane / 4, t = lane % 4;
                const int n = (g - OPC * q) & 7;             // phase output held by tile column g
                unsigned *o = &bv[((((size_t)ph * NR + q) * 32 + lane) * BW) * 4];
                if (mode == ws::MODE_BF16X3) {
                    // k slot 2t + 8 kq + e <-> chunk input 4t + 2 kq + e
                    for (int kq = 0; kq < 2; kq++) {
                        unsigned hi = 0, lo = 0;
                        for (int e = 0; e < 2; e++) {
                            const double v = bweight(rx, 4 * t + 2 * kq + e, n, xc0[ph], OP, bshift);
                            const unsigned short h = bf16_bits(v);
                            const unsigned short l = bf16_bits(v - bf16_value(h));
                            hi |= (unsigned)h << (16 * e);
                            lo |= (unsigned)l << (16 * e);
                        }
                        o[kq] = hi;
                        o[2 + kq] = lo;
                    }
                } else {
                    // velocities, TF32 MMA k2: slot t <-> input 4t + 2 k2, slot t + 4 <-> 4t + 2 k2 + 1
                    for (int k2 = 0; k2 < 2; k2++)
                        for (int e = 0; e < 2; e++) {
                            const double v = bweight(rx, 4 * t + 2 * k2 + e, n, xc0[ph], OP, bshift);
                            const unsigned h = tf32_bits(v);
                            o[4 * k2 + e] = h;
                            o[4 * k2 + 2 + e] = tf32_bits(v - tf32_value(h));
                        }
                }
                // products, FP16 MMA: k slots as the BF16 words
                unsigned *of = o + 4 * (BW - 1);
                for (int kq = 0; kq < 2; kq++) {
                    unsigned hi = 0, lo = 0;
                    for (int e = 0; e < 2; e++) {
                        const double v = bweight(rx, 4 * t + 2 * kq + e, n, xc0[ph], OP, bshift);
                        const unsigned short h = f16_bits(v);
                        const unsigned short l = f16_bits(v - f16_value(h));
                        hi |= (unsigned)h << (16 * e);
                        lo |= (unsigned)l << (16 * e);
                    }
                    of[kq] = hi;
                    of[2 + kq] = lo;
                }
            }
    cudaError_t e;
    if ((e = dev_malloc(&w.d_afrag, sizeof(unsigned) * zf.size())) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc z fragments");
    if ((e = cudaMemcpy(w.d_afrag, zf.data(), sizeof(unsigned) * zf.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "copy z fragments");
    if ((e = dev_malloc(&w.d_bvar, sizeof(unsigned) * bv.size())) != cudaSuccess) return cuda_fail(e, "cudaMalloc x fragments");
    if ((e = cudaMemcpy(w.d_bvar, bv.data(), sizeof(unsigned) * bv.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "copy x fragments");
    w.mode = mode;
    w.OP = OP;
    w.OPC = OPC;
    w.CB = CB;
    w.bshift = bshift;
    w.nchunk = (p->nlx - rx.dmin + bshift + CB - 1) / CB;
    for (int ph = 0; ph < 4; ph++) w.xc0[ph] = xc0[ph];
    w.KS = KS;
    w.zoff = zoff;
    w.ok = true;
    return EF_OK;
}

void ws_free(WsHost &w)
{
    cudaFree(w.d_afrag);
    cudaFree(w.d_bvar);
    w.d_afrag = nullptr;
    w.d_bvar = nullptr;
    w.ok = false;
}

cudaError_t ws_launch_bf16(const ws::WsMulti &m, int nz, int opc, cudaStream_t st);
cudaError_t ws_launch_tf32(const ws::WsMulti &m, int nz, int opc, cudaStream_t st);

// Kernel arguments of one plan for nsnap snapshots at u (the TMA view of u
// included), after the reference-profile launch on stream st.
static int ws_prepare(const ef_plan *p, int nsnap, const float *u, float *h, double *uref, double *plane_mean, int nf,
                      cudaStream_t st, ws::WsArgs *a)
{
    const WsHost &w = p->ws;
    memset(a, 0, sizeof *a);
    a->box_rows = p->nz > 256 ? p->nz / 2 : p->nz;
    int rc = encode_u_map(u, p->nx, p->ny, p->nz, nsnap, ws::CW, a->box_rows, &a->tmap);
    if (rc) return rc;
    // the reference profile first (1/nz of a plane read), then the persistent kernel
    ws_uref<<<dim3(p->ny, nsnap), 96, 0, st>>>(u, p->nx, p->ny, p->nz, uref, p->d_err);
    a->u = u; a->h = h; a->uref = uref; a->plane_mean = plane_mean; a->err = p->d_err;
    a->nx = p->nx; a->ny = p->ny; a->nz = p->nz; a->nlx = p->nlx; a->nlz = p->nlz;
    a->nchunk = w.nchunk; a->bshift = w.bshift; a->rx = p->rx.r; a->CB = w.CB; a->OP = w.OP;
    for (int ph = 0; ph < 4; ph++) a->xc0[ph] = w.xc0[ph];
    a->RZ = p->rz.r; a->KS = w.KS; a->zoff = w.zoff; a->nf = nf; a->nsnap = nsnap;
    a->wait_limit = p->wait_limit > 0 ? p->wait_limit : fz::kWaitCycles;
    a->afrag = reinterpret_cast<const uint4 *>(w.d_afrag);
    a->bvar = reinterpret_cast<const uint4 *>(w.d_bvar);
    return EF_OK;
}

static int ws_launch_class(const ws::WsMulti &m, int nz, int mode, int opc, cudaStream_t st)
{
    const cudaError_t e = mode == ws::MODE_TF32X2 ? ws_launch_tf32(m, nz, opc, st) : ws_launch_bf16(m, nz, opc, st);
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "xz_ws launch");
}

int ws_run(const ef_plan *p, int nsnap, const float *u, float *h, double *uref, double *plane_mean, int nf,
           cudaStream_t st)
{
    ws::WsMulti m;
    memset(&m, 0, sizeof m);
    m.nplan = 1;
    int rc = ws_prepare(p, nsnap, u, h, uref, plane_mean, nf, st, &m.plan[0]);
    if (rc) return rc;
    return ws_launch_class(m, p->nz, p->ws.mode, p->ws.OPC, st);
}

// The x-z stage of several plans (each with nsnap[i] snapshots at u[i] and
// its own scratch), one launch per kernel class (nz, precision, outputs per
// chunk) of at most kWsMaxPlans plans.  Every plan must run the
// warp-specialised kernel.
int ws_run_batch(ef_plan *const *plans, const int *nsnap, const float *const *u, int n, int nf, cudaStream_t st)
{
    std::vector<bool> done(n, false);
    for (int i = 0; i < n; i++) {
        if (done[i]) continue;
        const ef_plan *c = plans[i];
        ws::WsMulti m;
        memset(&m, 0, sizeof m);
        for (int k = i; k < n && m.nplan < ws::kWsMaxPlans; k++) {
            const ef_plan *q = plans[k];
            if (done[k] || q->nz != c->nz || q->ws.mode != c->ws.mode || q->ws.OPC != c->ws.OPC) continue;
            int rc = ws_prepare(q, nsnap[k], u[k], static_cast<float *>(q->d_h), q->d_uref, nullptr, nf, st,
                                &m.plan[m.nplan++]);
            if (rc) return rc;
            done[k] = true;
        }
        int rc = ws_launch_class(m, c->nz, c->ws.mode, c->ws.OPC, st);
        if (rc) return rc;
    }
    return EF_OK;
}

cudaError_t ws_launch_bf16(const ws::WsMulti &m, int nz, int opc, cudaStream_t st)
{
    using namespace ws;
#define ELES_WS_GO(NZ)                                                                                   \
    if (nz == NZ) return opc == 2 ? ws_launch<NZ, MODE_BF16X3, 2>(m, st) : ws_launch<NZ, MODE_BF16X3, 1>(m, st);
    ELES_WS_NZ_LIST(ELES_WS_GO)
#undef ELES_WS_GO
    return cudaErrorInvalidValue;
}

}  // namespace eles
