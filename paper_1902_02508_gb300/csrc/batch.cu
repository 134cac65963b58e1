// Batches of snapshots over several plans (different grids and filter
// widths) replayed as one CUDA graph, and a small autotuner that picks, per
// plan, the x-z kernel variant and the number of columns per z phase by
// timing them on a sample snapshot.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "eles_internal.h"

struct ef_batch {
    std::vector<ef_plan *> plans;
    std::vector<int> nsnap;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> key;   // pointers the graph was captured with
    std::vector<unsigned> gens;      // the plans' generations at capture
    long captures = 0;
    int device = 0;
};

using namespace eles;

namespace {

void drop_graph(ef_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->key.clear();
    b->gens.clear();
}

// The items' x-z stages: plans on the warp-specialised tensor-core kernel go
// through one persistent launch per kernel class (all their snapshots, grids
// and filter widths in one work list); the others run their own path.  Then
// every such plan's y stage.
int run_items(ef_batch *b, const void *const *u, void *const *ubar, void *const *tau, cudaStream_t s)
{
    std::vector<ef_plan *> wp;
    std::vector<int> wn;
    std::vector<const float *> wu;
    std::vector<size_t> wi;
    for (size_t i = 0; i < b->plans.size(); i++) {
        ef_plan *p = b->plans[i];
        if (p->fused && p->x_variant == 3 && p->ws.ok && b->nsnap[i] <= p->reserve) {
            wp.push_back(p);
            wn.push_back(b->nsnap[i]);
            wu.push_back(static_cast<const float *>(u[i]));
            wi.push_back(i);
            continue;
        }
        int rc = run_filter(p, b->nsnap[i], u[i], ubar[i], tau[i], nullptr, true, s, nullptr);
        if (rc) return rc;
    }
    if (!wp.empty()) {
        int rc = ws_run_batch(wp.data(), wn.data(), wu.data(), (int)wp.size(), 9, s);
        if (rc) return rc;
        for (size_t k = 0; k < wp.size(); k++)
            if ((rc = run_y_stage(wp[k], wn[k], ubar[wi[k]], tau[wi[k]], true, s))) return rc;
    }
    return EF_OK;
}

}  // namespace

extern "C" {

int ef_batch_create(ef_plan *const *plans, const int *nsnap, int n, ef_batch **out)
{
    if (!plans || !nsnap || n < 1 || !out) { set_error("ef_batch_create: bad arguments"); return EF_ERR_ARG; }
    *out = nullptr;
    for (int i = 0; i < n; i++) {
        if (!plans[i] || nsnap[i] < 1) { set_error("ef_batch_create: item %d invalid", i); return EF_ERR_ARG; }
        for (int k = 0; k < i; k++)
            if (plans[k] == plans[i]) { set_error("ef_batch_create: plan %d repeats plan %d (plans own scratch)", i, k); return EF_ERR_ARG; }
    }
    ef_batch *b = new ef_batch();
    cudaGetDevice(&b->device);
    for (int i = 0; i < n; i++) {
        int rc = plan_reserve(plans[i], nsnap[i]);
        if (rc) { delete b; return rc; }
        b->plans.push_back(plans[i]);
        b->nsnap.push_back(nsnap[i]);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete b; return cuda_fail(e, "ef_batch_create"); }
    *out = b;
    return EF_OK;
}

long ef_batch_captures(const ef_batch *b) { return b ? b->captures : -1; }

void ef_batch_destroy(ef_batch *b)
{
    if (!b) return;
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

int ef_batch_run(ef_batch *b, const void *const *u, void *const *ubar, void *const *tau, void *stream)
{
    if (!b || !u || !ubar || !tau) { set_error("ef_batch_run: NULL argument"); return EF_ERR_ARG; }
    const size_t n = b->plans.size();
    std::vector<const void *> key;
    for (size_t i = 0; i < n; i++) {
        if (!u[i] || !ubar[i] || !tau[i]) { set_error("ef_batch_run: NULL field of item %zu", i); return EF_ERR_ARG; }
        if (((uintptr_t)u[i]) % 16) { set_error("ef_batch_run: u of item %zu not 16-byte aligned", i); return EF_ERR_ARG; }
        key.push_back(u[i]); key.push_back(ubar[i]); key.push_back(tau[i]);
    }
    std::vector<unsigned> gens;
    for (ef_plan *p : b->plans) gens.push_back(p->gen);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!b->exec || key != b->key || gens != b->gens) {
        drop_graph(b);
        // one eager pass (first-use kernel attributes are set outside capture)
        int rc = run_items(b, u, ubar, tau, b->cap);
        if (rc) return rc;
        if ((e = cudaStreamSynchronize(b->cap)) != cudaSuccess) return cuda_fail(e, "ef_batch_run");
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "begin capture");
        rc = run_items(b, u, ubar, tau, b->cap);
        e = cudaStreamEndCapture(b->cap, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { b->exec = nullptr; return cuda_fail(e, "graph instantiate"); }
        b->key = key;
        b->gens = gens;
        b->captures++;
    }
    if ((e = cudaGraphLaunch(b->exec, s)) != cudaSuccess) return cuda_fail(e, "graph launch");
    return EF_OK;
}

// Try the x-z variants the plan supports and keep the fastest.  u: one
// sample snapshot on the device in the plan's precision; ubar/tau scratch
// outputs.  *choice receives the variant (0 unfused, 1 fused CUDA cores,
// 2 fused tensor cores, 3 fused tensor cores, warp-specialised) * 16 + P.
// Synchronises the device.
int ef_plan_autotune(ef_plan *p, const void *u, void *ubar, void *tau, int reps, int *choice, float *best_ms)
{
    if (!p || !u || !ubar || !tau) { set_error("ef_plan_autotune: NULL argument"); return EF_ERR_ARG; }
    if (p->diff) { set_error("ef_plan_autotune: the differential filter has one variant"); return EF_ERR_UNSUPPORTED; }
    if (reps < 1) reps = 3;
    p->gen++;
    struct Cand { bool fused; int xv; int P; };
    std::vector<Cand> cands;
    const Cand orig = {p->fused, p->x_variant, p->P};
    cands.push_back({false, p->rx.ok ? 1 : 0, p->P});
    if (orig.fused) {
        if (p->ws.ok) cands.push_back({true, 3, p->P});
        for (int xv = 1; xv <= 2; xv++) {
            if (xv == 2 && !p->tc_ok) continue;
            if (xv == 1 && (!fused_supported(p->rx.r, p->rx.D, p->rz.r, p->rz.D) || !p->nblk_x)) continue;
            for (int P = 2; P <= 8; P *= 2) {
                const size_t need = xv == 2 ? tc_smem_bytes(P, p->nz, p->tc.KS) : fused_smem_bytes(p->rx.r, P, p->nz);
                if (need <= 222 * 1024) cands.push_back({true, xv, P});
            }
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Cand win = orig;
    int rc = EF_OK;
    for (const Cand &c : cands) {
        p->fused = c.fused;
        p->x_variant = c.xv;
        p->P = c.P;
        if (!p->fused && !p->d_g) {   // the unfused path needs its x scratch
            const size_t es = p->prec == EF_PREC_FP64 ? sizeof(double) : sizeof(float);
            cudaError_t e = dev_malloc(&p->d_g, es * 9 * (size_t)p->ny * p->nz * p->nlx);
            if (e != cudaSuccess) { rc = cuda_fail(e, "autotune scratch"); break; }
        }
        if (p->fused) {
            int NQ = 1;
            for (int q = p->nz / (9 * p->P); q > 1; q--)
                if (p->nlz % q == 0) { NQ = q; break; }
            p->NQ = NQ;
            p->ZQs = p->nlz / NQ;
        }
        rc = run_filter(p, 1, u, ubar, tau, nullptr, true, nullptr, nullptr);   // warm-up
        if (rc) break;
        cudaEventRecord(e0);
        for (int r = 0; r < reps && !rc; r++) rc = run_filter(p, 1, u, ubar, tau, nullptr, true, nullptr, nullptr);
        cudaEventRecord(e1);
        cudaError_t e = cudaEventSynchronize(e1);
        if (rc) break;
        if (e != cudaSuccess) { rc = cuda_fail(e, "autotune timing"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < best) { best = ms; win = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->fused = win.fused;
    p->x_variant = win.xv;
    p->P = win.P;
    if (p->fused) {
        int NQ = 1;
        for (int q = p->nz / (9 * p->P); q > 1; q--)
            if (p->nlz % q == 0) { NQ = q; break; }
        p->NQ = NQ;
        p->ZQs = p->nlz / NQ;
    }
    if (rc) return rc;
    if (choice) *choice = (win.fused ? win.xv : 0) * 16 + win.P;
    if (best_ms) *best_ms = best;
    return EF_OK;
}

// Apply a choice made earlier (for example one read from a tuning cache).
static int set_x_variant(ef_plan *p, int choice)
{
    const int v = choice / 16, P = choice % 16;
    if (P < 1 || (P & (P - 1)) || P > 8) { set_error("ef_plan_set_variant: bad column count"); return EF_ERR_ARG; }
    if (v == 0) {
        if (!p->d_g) {
            const size_t es = p->prec == EF_PREC_FP64 ? sizeof(double) : sizeof(float);
            cudaError_t e = dev_malloc(&p->d_g, es * 9 * (size_t)p->ny * p->nz * p->nlx);
            if (e != cudaSuccess) return cuda_fail(e, "ef_plan_set_variant");
        }
        p->fused = false;
        p->x_variant = p->rx.ok ? 1 : 0;
        return EF_OK;
    }
    if (v == 3) {
        if (!p->ws.ok) { set_error("ef_plan_set_variant: warp-specialised kernel unavailable"); return EF_ERR_UNSUPPORTED; }
        p->fused = true;
        p->x_variant = 3;
        return EF_OK;
    }
    if (v > 3) { set_error("ef_plan_set_variant: unknown variant %d", v); return EF_ERR_ARG; }
    if (v == 2 && !p->tc_ok) { set_error("ef_plan_set_variant: tensor cores unavailable"); return EF_ERR_UNSUPPORTED; }
    if (v == 1 && !fused_supported(p->rx.r, p->rx.D, p->rz.r, p->rz.D)) { set_error("ef_plan_set_variant: fused kernel unavailable"); return EF_ERR_UNSUPPORTED; }
    const size_t need = v == 2 ? tc_smem_bytes(P, p->nz, p->tc.KS) : fused_smem_bytes(p->rx.r, P, p->nz);
    if (need > 222 * 1024 || !p->nblk_x) { set_error("ef_plan_set_variant: variant does not fit this grid"); return EF_ERR_UNSUPPORTED; }
    p->fused = true;
    p->x_variant = v;
    p->P = P;
    int NQ = 1;
    for (int q = p->nz / (9 * p->P); q > 1; q--)
        if (p->nlz % q == 0) { NQ = q; break; }
    p->NQ = NQ;
    p->ZQs = p->nlz / NQ;
    return EF_OK;
}

int ef_plan_set_variant(ef_plan *p, int choice)
{
    if (!p) { set_error("ef_plan_set_variant: NULL plan"); return EF_ERR_ARG; }
    if (p->diff) { set_error("ef_plan_set_variant: the differential filter has one variant"); return EF_ERR_UNSUPPORTED; }
    const bool split = p->prec == EF_PREC_BF16X3 || p->prec == EF_PREC_TF32X2;
    if ((choice & EF_VARIANT_CUDA_CORE_Y) && !split) {
        set_error("ef_plan_set_variant: only split-precision plans have a y choice");
        return EF_ERR_ARG;
    }
    const int rc = set_x_variant(p, choice & (EF_VARIANT_CUDA_CORE_Y - 1));
    if (rc) return rc;
    p->ytc_ok = p->ytc_fit && !(choice & EF_VARIANT_CUDA_CORE_Y);
    p->gen++;
    return EF_OK;
}

}  // extern "C"
