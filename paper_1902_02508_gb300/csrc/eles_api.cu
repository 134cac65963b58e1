// The C ABI of include/eles.h: argument checks, plan lifetime, dispatch.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "eles_internal.h"
#include "fused_stage.cuh"

namespace eles {

static thread_local char g_msg[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
}

static std::atomic<int> g_fail_alloc{-1};   // allocations to let through before one fails (-1: none fails)

static bool alloc_should_fail()
{
    int n = g_fail_alloc.load();
    while (n >= 0) {
        if (g_fail_alloc.compare_exchange_weak(n, n - 1)) return n == 0;
    }
    return false;
}

cudaError_t dev_malloc_void(void **p, size_t bytes)
{
    if (alloc_should_fail()) { *p = nullptr; return cudaErrorMemoryAllocation; }
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async_void(void **p, size_t bytes, cudaStream_t s)
{
    if (alloc_should_fail()) { *p = nullptr; return cudaErrorMemoryAllocation; }
    return cudaMallocAsync(p, bytes, s);
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
}

static void free_band(Band &b)
{
    cudaFree(b.d_start);
    cudaFree(b.d_w64);
    cudaFree(b.d_w32);
    b = Band();
}

static int check_grid(const ef_grid *g, const char *name)
{
    if (!g || !g->y) { set_error("%s: NULL grid or y", name); return EF_ERR_ARG; }
    if (g->nx < 1 || g->ny < 3 || g->nz < 1) { set_error("%s: sizes must be nx,nz >= 1, ny >= 3", name); return EF_ERR_SHAPE; }
    if (!(g->Lx > 0) || !(g->Lz > 0)) { set_error("%s: Lx, Lz must be > 0", name); return EF_ERR_ARG; }
    if (g->y[0] != -1.0 || g->y[g->ny - 1] != 1.0) { set_error("%s: y must run from -1 to +1", name); return EF_ERR_ARG; }
    for (int j = 1; j < g->ny; j++)
        if (!(g->y[j] > g->y[j - 1])) { set_error("%s: y must be strictly ascending", name); return EF_ERR_ARG; }
    return EF_OK;
}

}  // namespace eles

namespace eles {

// Accumulate a finished slot's phase times into the plan's totals.
static int prof_collect(ef_plan *p, int slot)
{
    if (!p->prof_used[slot]) return EF_OK;
    cudaError_t e = cudaEventSynchronize(p->prof_ev[slot][ef_plan::kProfEvents - 1]);
    if (e != cudaSuccess) return cuda_fail(e, "profile events");
    for (int k = 0; k < 4; k++) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, p->prof_ev[slot][k], p->prof_ev[slot][k + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "profile events");
        p->prof_ms[k] += ms;
    }
    p->prof_used[slot] = false;
    p->prof_calls++;
    return EF_OK;
}

int prof_begin(ef_plan *p, PhaseEvents *pe)
{
    const int slot = (int)((p->prof_calls + 0) % ef_plan::kProfSlots);
    int free_slot = -1;
    for (int t = 0; t < ef_plan::kProfSlots; t++)
        if (!p->prof_used[(slot + t) % ef_plan::kProfSlots]) { free_slot = (slot + t) % ef_plan::kProfSlots; break; }
    if (free_slot < 0) {
        for (int t = 0; t < ef_plan::kProfSlots; t++) {
            int rc = prof_collect(p, t);
            if (rc) return rc;
        }
        free_slot = 0;
    }
    for (int k = 0; k < ef_plan::kProfEvents; k++) {
        if (!p->prof_ev[free_slot][k]) {
            cudaError_t e = cudaEventCreate(&p->prof_ev[free_slot][k]);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        }
        pe->e[k] = p->prof_ev[free_slot][k];
    }
    p->prof_used[free_slot] = true;
    return EF_OK;
}

// (Re)allocate the plan's scratch for batches of up to nsnap snapshots.
int plan_reserve(ef_plan *p, int nsnap)
{
    if (nsnap < 1) { set_error("reserve: nsnap must be >= 1"); return EF_ERR_ARG; }
    if (p->diff) {                  // the differential filter runs snapshots one after another
        if (nsnap > p->reserve) p->reserve = nsnap;
        return EF_OK;
    }
    if (nsnap <= p->reserve) return EF_OK;
    p->gen++;   // the scratch pointers change: graphs holding the old ones are stale
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "reserve");
    cudaFree(p->d_g); cudaFree(p->d_h); cudaFree(p->d_uref); cudaFree(p->d_urefT); cudaFree(p->d_rowsum);
    cudaFree(p->d_AU); cudaFree(p->d_AUU); cudaFree(p->d_wy); cudaFree(p->d_ytmp); cudaFree(p->d_yfrag);
    cudaFree(p->d_Kab);
    p->d_Kab = nullptr;
    p->d_g = p->d_h = p->d_urefT = p->d_wy = p->d_ytmp = nullptr;
    p->d_yfrag = nullptr;
    p->d_uref = p->d_rowsum = p->d_AU = p->d_AUU = nullptr;
    p->reserve = 0;
    const size_t es = (p->prec == EF_PREC_FP64) ? sizeof(double) : sizeof(float);
    const size_t S = (size_t)nsnap;
    struct { void **ptr; size_t bytes; } req[] = {
        {&p->d_g, p->fused ? 0 : es * 9 * (size_t)p->ny * p->nz * p->nlx},
        {&p->d_h, es * 9 * S * p->ny * p->nlz * p->nlx},
        {(void **)&p->d_uref, sizeof(double) * 3 * S * p->ny},
        {&p->d_urefT, es * 3 * (size_t)p->ny},
        {(void **)&p->d_rowsum, sizeof(double) * 3 * (size_t)p->ny * p->nzw},
        {(void **)&p->d_AU, sizeof(double) * 3 * S * p->nly},
        {(void **)&p->d_AUU, sizeof(double) * 6 * S * p->nly},
        {(void **)&p->d_Kab, sizeof(float) * 6 * S * p->nly},
        {&p->d_wy, es * 8 * S * p->nly * p->ny},
        {&p->d_ytmp, es * kYTmp * S * p->nly * p->nlz * p->nlx},
        {(void **)&p->d_yfrag, p->ytc_ok ? sizeof(uint4) * kYOps * 64 * S * p->ytc.kstot : 0},
    };
    for (auto &r : req) {
        if (!r.bytes) continue;
        e = dev_malloc(r.ptr, r.bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc scratch");
    }
    p->reserve = nsnap;
    return EF_OK;
}

}  // namespace eles

using namespace eles;

extern "C" {

const char *ef_last_error(void) { return g_msg; }

const char *ef_version(void)
{
#ifdef ELES_CHECK
    return "eles-gb300 0.2 (sm_103a, range-checked build)";
#else
    return "eles-gb300 0.2 (sm_103a)";
#endif
}

int ef_debug_fail_alloc(int n)
{
    if (n < -1) { set_error("ef_debug_fail_alloc: n must be >= -1"); return EF_ERR_ARG; }
    g_fail_alloc.store(n);
    return EF_OK;
}

void ef_plan_destroy(ef_plan *p)
{
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    free_band(p->bx);
    free_band(p->bz);
    cudaFree(p->d_ystart);
    cudaFree(p->d_ycount);
    for (int q = 0; q < 2; q++) { cudaFree(p->d_yw64[q]); cudaFree(p->d_yw32[q]); }
    cudaFree(p->d_ygrid);
    cudaFree(p->d_g);
    cudaFree(p->d_h);
    cudaFree(p->d_uref);
    cudaFree(p->d_urefT);
    cudaFree(p->d_rowsum);
    cudaFree(p->d_AU);
    cudaFree(p->d_AUU);
    cudaFree(p->d_Kab);
    cudaFree(p->d_wy);
    cudaFree(p->d_ytmp);
    cudaFree(p->d_yfrag);
    cudaFree(p->d_zfrag);
    ws_free(p->ws);
    cudaFree(p->d_err);
    diff_destroy(p->diff);
    for (int t = 0; t < ef_plan::kProfSlots; t++)
        for (int k = 0; k < ef_plan::kProfEvents; k++)
            if (p->prof_ev[t][k]) cudaEventDestroy(p->prof_ev[t][k]);
    cudaSetDevice(cur);
    delete p;
}

int ef_filter_setup(const ef_grid *dns, const ef_grid *les, double delta, int kernel, int extension,
                    int precision, ef_plan **out)
{
    if (!out) { set_error("ef_filter_setup: out is NULL"); return EF_ERR_ARG; }
    *out = nullptr;
    int rc;
    if ((rc = check_grid(dns, "dns")) || (rc = check_grid(les, "les"))) return rc;
    if (!(delta > 0) || !isfinite(delta)) { set_error("delta must be finite and > 0"); return EF_ERR_ARG; }
    if (kernel != EF_KERNEL_GAUSSIAN && kernel != EF_KERNEL_GAUSSIAN_HAT && kernel != EF_KERNEL_DIFFERENTIAL) {
        set_error("unknown filter kernel %d", kernel);
        return EF_ERR_UNSUPPORTED;
    }
    const bool differential = kernel == EF_KERNEL_DIFFERENTIAL;
    if (extension < EF_EXT_EVEN_ODD || extension > EF_EXT_NONE) { set_error("unknown extension %d", extension); return EF_ERR_ARG; }
    if (precision != EF_PREC_FP64 && precision != EF_PREC_FP32 && precision != EF_PREC_BF16X3 &&
        precision != EF_PREC_TF32X2) {
        set_error("unknown precision %d", precision);
        return EF_ERR_UNSUPPORTED;
    }
    const bool split = precision == EF_PREC_BF16X3 || precision == EF_PREC_TF32X2;
    if (split && kernel == EF_KERNEL_DIFFERENTIAL) {
        set_error("the differential filter runs in FP64 or FP32 (EF_PREC_FP64, EF_PREC_FP32)");
        return EF_ERR_UNSUPPORTED;
    }
    if (les->Lx != dns->Lx || les->Lz != dns->Lz) { set_error("LES and DNS boxes differ"); return EF_ERR_SHAPE; }
    if (les->nx > dns->nx || les->nz > dns->nz || les->ny > dns->ny) { set_error("LES grid finer than DNS grid"); return EF_ERR_SHAPE; }
    if (!differential && (2.5 * delta >= 0.5 * dns->Lx || 2.5 * delta >= 0.5 * dns->Lz || 2.5 * delta >= 2.0)) {
        set_error("filter support 2.5 delta must be below half of Lx, Lz and below 2");
        return EF_ERR_ARG;
    }
    ef_plan *p = new ef_plan();
    cudaGetDevice(&p->device);
    p->nx = dns->nx; p->ny = dns->ny; p->nz = dns->nz;
    p->nlx = les->nx; p->nly = les->ny; p->nlz = les->nz;
    p->Lx = dns->Lx; p->Lz = dns->Lz; p->delta = delta;
    p->ext = extension; p->prec = precision;
    p->yquad = kernel == EF_KERNEL_GAUSSIAN_HAT ? 1 : 0;
    if (extension == EF_EXT_ODD_EVEN) { p->par[0] = -1; p->par[1] = 1; p->par[2] = -1; }
    cudaError_t e;
#define CK(x, what) do { if ((e = (x)) != cudaSuccess) { rc = cuda_fail(e, what); goto fail; } } while (0)
    if (differential) {
        if ((rc = diff_setup(p, dns->y, les->y))) goto fail;
        p->reserve = 1;
        CK(dev_malloc(&p->d_err, sizeof(int)), "cudaMalloc error word");
        CK(cudaMemset(p->d_err, 0, sizeof(int)), "clear error word");
        CK(cudaDeviceSynchronize(), "setup");
    } else {
        CK(dev_malloc(&p->d_ygrid, sizeof(double) * p->ny), "cudaMalloc y");
        CK(cudaMemcpy(p->d_ygrid, dns->y, sizeof(double) * p->ny, cudaMemcpyHostToDevice), "copy y");
        if ((rc = build_periodic_band(p->nx, p->Lx, p->nlx, delta, &p->bx))) goto fail;
        if ((rc = build_periodic_band(p->nz, p->Lz, p->nlz, delta, &p->bz))) goto fail;
        if ((rc = build_wall_rows(p, les->y))) goto fail;
        CK(cudaDeviceSynchronize(), "operator kernels");
        if ((rc = build_ring(p->bx, &p->rx))) goto fail;
        if ((rc = build_ring(p->bz, &p->rz))) goto fail;
        p->x_variant = p->rx.ok ? 1 : 0;
        // FP32 plans use the fused x-z kernel when its ring sizes are instantiated
        // (CUDA cores); BF16X3 may also run the tensor-core fused kernel (variant 2)
        const bool tc = precision == EF_PREC_BF16X3 && p->rx.ok && p->rz.ok &&
                        tc_supported(p->rx.r, p->rx.D, p->rz.r, p->rz.D, p->nlz);
        if (precision != EF_PREC_FP64 && p->rx.ok && p->rz.ok && p->nz <= kFusedMaxRows && p->nz % 32 == 0 &&
            (tc || fused_supported(p->rx.r, p->rx.D, p->rz.r, p->rz.D)) &&
            p->nlx % fused_stage_blocks(p->rx.r) == 0) {
            const int SB = fused_stage_blocks(p->rx.r);
            std::vector<unsigned> zf;
            int zoff = 0;
            const int KS = tc ? tc_zfrags(p->rz, p->nlz, zf, &zoff) : 0;
            auto smem = [&](int P) {
                return tc ? tc_smem_bytes(P, p->nz, KS) : fused_smem_bytes(p->rx.r, P, p->nz);
            };
            p->P = 8;
            while (p->P > 1 && smem(p->P) > 222 * 1024) p->P /= 2;
            if (smem(p->P) <= 222 * 1024) {
                p->fused = true;
                p->NQ = 1;
                for (int q = p->nz / (9 * p->P); q > 1; q--)
                    if (p->nlz % q == 0) { p->NQ = q; break; }
                p->ZQs = p->nlz / p->NQ;
                // stream start: dmax rounded up to whole stages, so no stage wraps and
                // every stage starts on a 16-byte boundary
                p->bshift = (p->rx.dmax + SB - 1) / SB * SB;
                const int need = p->nlx - p->rx.dmin + p->bshift;
                p->nblk_x = (need + SB - 1) / SB * SB;
                if (tc) {
                    p->tc_ok = true;
                    p->x_variant = 2;
                    tc_weights(p->rx, &p->tc);
                    p->tc.KS = KS;
                    p->tc.zoff = zoff;
                    if (KS > 0) {
                        CK(dev_malloc(&p->d_zfrag, sizeof(unsigned) * zf.size()), "cudaMalloc z fragments");
                        CK(cudaMemcpy(p->d_zfrag, zf.data(), sizeof(unsigned) * zf.size(), cudaMemcpyHostToDevice),
                           "copy z fragments");
                        p->tc.afrag = p->d_zfrag;
                    }
                }
            }
        }
        if (split) {
            // the warp-specialised tensor-core kernel; a split-precision plan never
            // falls back to CUDA-core contractions by itself
            const char *why = nullptr;
            if ((rc = ws_setup(p, &why))) goto fail;
            if (p->ws.ok) {
                p->fused = true;
                p->x_variant = 3;
            } else if (!p->tc_ok) {
                set_error("ef_filter_setup: no tensor-core x-z kernel for this plan (%s)", why ? why : "unsupported");
                rc = EF_ERR_UNSUPPORTED;
                goto fail;
            }
        }
        p->nzw = (p->nz + 31) / 32;
        if ((rc = plan_reserve(p, 1))) goto fail;
        CK(dev_malloc(&p->d_err, sizeof(int)), "cudaMalloc error word");
        CK(cudaMemset(p->d_err, 0, sizeof(int)), "clear error word");
        CK(cudaDeviceSynchronize(), "setup");
    }
#undef CK
    *out = p;
    return EF_OK;
fail:
    ef_plan_destroy(p);
    return rc;
}


static int hot_args(ef_plan *p, const void *u, const void *ubar, const char *who)
{
    if (!p || !u || !ubar) { set_error("%s: NULL plan or field pointer", who); return EF_ERR_ARG; }
    if (((uintptr_t)u) % 16) { set_error("%s: u must be 16-byte aligned", who); return EF_ERR_ARG; }
    return EF_OK;
}

int ef_plan_set_wait_limit(ef_plan *p, long long cycles)
{
    if (!p || cycles < 0) { set_error("ef_plan_set_wait_limit: NULL plan or negative limit"); return EF_ERR_ARG; }
    p->wait_limit = cycles;
    p->gen++;   // batch graphs hold the limit in their launch arguments
    return EF_OK;
}

int ef_plan_reserve(ef_plan *p, int max_snapshots)
{
    if (!p) { set_error("ef_plan_reserve: NULL plan"); return EF_ERR_ARG; }
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    int rc = plan_reserve(p, max_snapshots);
    cudaSetDevice(cur);
    return rc;
}

int ef_filter_fields(ef_plan *p, const void *u, void *ubar, void *stream)
{
    NvtxRange nv("ef_filter_fields");
    int rc = hot_args(p, u, ubar, "ef_filter_fields");
    if (rc) return rc;
    PhaseEvents pe;
    if (p->prof_on && (rc = prof_begin(p, &pe))) return rc;
    return run_filter(p, 1, u, ubar, nullptr, nullptr, false, static_cast<cudaStream_t>(stream),
                      p->prof_on ? &pe : nullptr);
}

int ef_subfilter_stress_batch(ef_plan *p, int nsnap, const void *u, void *ubar, void *tau, double *plane_mean,
                              void *stream)
{
    NvtxRange nv("ef_subfilter_stress");
    int rc = hot_args(p, u, ubar, "ef_subfilter_stress");
    if (rc) return rc;
    if (!tau) { set_error("ef_subfilter_stress: tau is NULL"); return EF_ERR_ARG; }
    if (nsnap < 1) { set_error("ef_subfilter_stress_batch: nsnap must be >= 1"); return EF_ERR_ARG; }
    PhaseEvents pe;
    if (p->prof_on && (rc = prof_begin(p, &pe))) return rc;
    return run_filter(p, nsnap, u, ubar, tau, plane_mean, true, static_cast<cudaStream_t>(stream),
                      p->prof_on ? &pe : nullptr);
}

int ef_subfilter_stress(ef_plan *p, const void *u, void *ubar, void *tau, double *plane_mean, void *stream)
{
    return ef_subfilter_stress_batch(p, 1, u, ubar, tau, plane_mean, stream);
}

int ef_profile_enable(ef_plan *p, int on)
{
    if (!p) { set_error("ef_profile_enable: NULL plan"); return EF_ERR_ARG; }
    if (on) {
        for (int t = 0; t < ef_plan::kProfSlots; t++) p->prof_used[t] = false;
        p->prof_calls = 0;
        for (int k = 0; k < 4; k++) p->prof_ms[k] = 0.0;
    }
    p->prof_on = on != 0;
    return EF_OK;
}

int ef_profile_read(ef_plan *p, double *ms, long *calls)
{
    if (!p || !ms) { set_error("ef_profile_read: NULL argument"); return EF_ERR_ARG; }
    for (int t = 0; t < ef_plan::kProfSlots; t++) {
        int rc = prof_collect(p, t);
        if (rc) return rc;
    }
    for (int k = 0; k < 4; k++) ms[k] = p->prof_ms[k];
    if (calls) *calls = p->prof_calls;
    return EF_OK;
}

// Failure-detection self-test: thread 0 waits on an mbarrier with the
// bounded wait every kernel of the library uses.  With complete = 0 nothing
// arrives on it, so the wait gives up after `limit` SM clocks and records
// EF_ERR_TIMEOUT in the error word; with complete = 1 the phase completes
// first and nothing is recorded.  No copy is in flight and no TMEM is held.
namespace {
__global__ void selftest_wait_kernel(int *err, long long limit, int complete)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x != 0) return;
    fz::mbar_init(&bar, 1);
    fz::mbar_fence_init();
    if (complete) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(fz::smem_u32(&bar)) : "memory");
    fz::mbar_wait_for(&bar, 0, err, limit);
}
}  // namespace

int ef_selftest_wait(ef_plan *p, long long limit_cycles, int complete, void *stream)
{
    if (!p) { set_error("ef_selftest_wait: NULL plan"); return EF_ERR_ARG; }
    if (limit_cycles < 1 || limit_cycles > 4000000000LL) {
        set_error("ef_selftest_wait: limit must be 1 .. 4e9 SM clocks");
        return EF_ERR_ARG;
    }
    selftest_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(p->d_err, limit_cycles, complete ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "ef_selftest_wait");
}

int ef_check_device_error(ef_plan *p, void *stream)
{
    if (!p) { set_error("ef_check_device_error: NULL plan"); return EF_ERR_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int code = 0;
    cudaError_t e = cudaMemcpyAsync(&code, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_err, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "read device error word");
    if (code) set_error("device reported status %d", code);
    return code;
}

int ef_plan_info(const ef_plan *p, int what, long *value)
{
    if (!p || !value) { set_error("ef_plan_info: NULL argument"); return EF_ERR_ARG; }
    switch (what) {
    case 0: *value = p->nx; break;
    case 1: *value = p->ny; break;
    case 2: *value = p->nz; break;
    case 3: *value = p->nlx; break;
    case 4: *value = p->nly; break;
    case 5: *value = p->nlz; break;
    case 6: *value = p->prec; break;
    case 7: *value = p->rx.ok ? 2 * p->rx.R + 1 : p->bx.T; break;
    case 8: *value = p->rz.ok ? 2 * p->rz.R + 1 : p->bz.T; break;
    case 9: *value = p->ytaps_max; break;
    case 10: *value = p->x_variant; break;
    case 11: *value = p->fused ? 1 : 0; break;
    case 12: *value = p->reserve; break;
    case 13: *value = p->ytc_ok ? 1 : 0; break;
    case 15: *value = p->x_variant == 3 ? p->ws.OP : 0; break;
    case 14: *value = p->diff ? 1 : 0; break;
    default: set_error("ef_plan_info: unknown index %d", what); return EF_ERR_ARG;
    }
    return EF_OK;
}

int ef_plan_weights(const ef_plan *p, int which, double *dst)
{
    if (!p || !dst) { set_error("ef_plan_weights: NULL argument"); return EF_ERR_ARG; }
    if (p->diff) { set_error("ef_plan_weights: the differential filter has no banded operators"); return EF_ERR_UNSUPPORTED; }
    cudaError_t e;
    if (which == 0 || which == 1) {
        const Band &b = which == 0 ? p->bx : p->bz;
        std::vector<double> w((size_t)b.nl * b.T);
        std::vector<int> st(b.nl);
        e = cudaMemcpy(w.data(), b.d_w64, sizeof(double) * w.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(st.data(), b.d_start, sizeof(int) * b.nl, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "ef_plan_weights");
        memset(dst, 0, sizeof(double) * (size_t)b.nl * b.n);
        for (int r = 0; r < b.nl; r++)
            for (int t = 0; t < b.T; t++) dst[(size_t)r * b.n + (st[r] + t) % b.n] += w[(size_t)r * b.T + t];
        return EF_OK;
    }
    if (which == 2 || which == 3) {
        e = cudaMemcpy(dst, p->d_yw64[which - 2], sizeof(double) * (size_t)p->nly * p->ny, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "ef_plan_weights");
        return EF_OK;
    }
    set_error("ef_plan_weights: unknown operator %d", which);
    return EF_ERR_ARG;
}

}  // extern "C"
