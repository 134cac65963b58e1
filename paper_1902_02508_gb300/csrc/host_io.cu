// Subfilter stress on host buffers: the copies of one group of snapshots in
// and of another group's results out overlap the compute of a third.
//
// A pipeline owns two device slots of `chunk` snapshots (the input field and
// the outputs), a copy-in and a copy-out stream, and events.  Group c uses
// slot c % 2:
//   copy-in stream   wait(compute of group c-2 done) -> H2D u      -> in[s]
//   compute stream   wait(in[s]) wait(out of group c-2 done) -> run -> comp[s]
//   copy-out stream  wait(comp[s]) -> D2H ubar, tau (, plane means) -> out[s]
// Each call starts both copy streams behind the caller's stream and ends with
// the caller's stream waiting on the last copies out, so calls on one stream
// are ordered and synchronising the caller's stream waits for everything.
#include <string.h>

#include "eles_internal.h"

struct ef_io {
    ef_plan *plan = nullptr;
    int chunk = 0;
    void *u[2] = {nullptr, nullptr}, *ubar[2] = {nullptr, nullptr}, *tau[2] = {nullptr, nullptr};
    double *pm[2] = {nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t start = nullptr, ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {};
};

using namespace eles;

namespace {

void release(ef_io *io)
{
    for (int k = 0; k < 2; k++) {
        cudaFree(io->u[k]); cudaFree(io->ubar[k]); cudaFree(io->tau[k]); cudaFree(io->pm[k]);
        if (io->ev_in[k]) cudaEventDestroy(io->ev_in[k]);
        if (io->ev_comp[k]) cudaEventDestroy(io->ev_comp[k]);
        if (io->ev_out[k]) cudaEventDestroy(io->ev_out[k]);
    }
    if (io->start) cudaEventDestroy(io->start);
    if (io->s_in) cudaStreamDestroy(io->s_in);
    if (io->s_out) cudaStreamDestroy(io->s_out);
    delete io;
}

}  // namespace

extern "C" {

int ef_io_create(ef_plan *p, int chunk, ef_io **out)
{
    if (!p || !out || chunk < 1) { set_error("ef_io_create: bad arguments"); return EF_ERR_ARG; }
    *out = nullptr;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    int rc = plan_reserve(p, chunk);
    if (rc) { cudaSetDevice(cur); return rc; }
    ef_io *io = new ef_io();
    io->plan = p;
    io->chunk = chunk;
    const size_t es = p->prec == EF_PREC_FP64 ? sizeof(double) : sizeof(float);
    const size_t nu = es * 3 * (size_t)p->nx * p->ny * p->nz * chunk;
    const size_t nl = (size_t)p->nlx * p->nly * p->nlz * chunk;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        e = dev_malloc(&io->u[k], nu);
        if (e == cudaSuccess) e = dev_malloc(&io->ubar[k], es * 3 * nl);
        if (e == cudaSuccess) e = dev_malloc(&io->tau[k], es * 6 * nl);
        if (e == cudaSuccess) e = dev_malloc((void **)&io->pm[k], sizeof(double) * 3 * p->ny * chunk);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->ev_in[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->ev_comp[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->ev_out[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io->s_out, cudaStreamNonBlocking);
    cudaSetDevice(cur);
    if (e != cudaSuccess) {
        release(io);
        return cuda_fail(e, "ef_io_create");
    }
    *out = io;
    return EF_OK;
}

void ef_io_destroy(ef_io *io)
{
    if (!io) return;
    cudaStreamSynchronize(io->s_in);
    cudaStreamSynchronize(io->s_out);
    release(io);
}

int ef_subfilter_stress_host(ef_io *io, int nsnap, const void *u_host, void *ubar_host, void *tau_host,
                             double *plane_mean_host, void *stream)
{
    if (!io || !u_host || !ubar_host || !tau_host) {
        set_error("ef_subfilter_stress_host: NULL argument");
        return EF_ERR_ARG;
    }
    if (nsnap < 1) { set_error("ef_subfilter_stress_host: nsnap must be >= 1"); return EF_ERR_ARG; }
    ef_plan *p = io->plan;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t es = p->prec == EF_PREC_FP64 ? sizeof(double) : sizeof(float);
    const size_t bu = es * 3 * (size_t)p->nx * p->ny * p->nz;       // bytes per snapshot
    const size_t nl = (size_t)p->nlx * p->nly * p->nlz;
    const size_t bb = es * 3 * nl, bt = es * 6 * nl, bp = sizeof(double) * 3 * p->ny;
    cudaError_t e;
#define CKE(x, what) do { if ((e = (x)) != cudaSuccess) return cuda_fail(e, what); } while (0)
    CKE(cudaEventRecord(io->start, s), "host io: start");
    CKE(cudaStreamWaitEvent(io->s_in, io->start, 0), "host io: order copy-in");
    CKE(cudaStreamWaitEvent(io->s_out, io->start, 0), "host io: order copy-out");
    const int ngroups = (nsnap + io->chunk - 1) / io->chunk;
    for (int c = 0; c < ngroups; c++) {
        const int k = c & 1, s0 = c * io->chunk;
        const int ns = nsnap - s0 < io->chunk ? nsnap - s0 : io->chunk;
        if (c >= 2) CKE(cudaStreamWaitEvent(io->s_in, io->ev_comp[k], 0), "host io: slot input free");
        CKE(cudaMemcpyAsync(io->u[k], static_cast<const char *>(u_host) + s0 * bu, ns * bu, cudaMemcpyHostToDevice,
                            io->s_in), "host io: copy in");
        CKE(cudaEventRecord(io->ev_in[k], io->s_in), "host io: input landed");
        CKE(cudaStreamWaitEvent(s, io->ev_in[k], 0), "host io: wait input");
        if (c >= 2) CKE(cudaStreamWaitEvent(s, io->ev_out[k], 0), "host io: slot outputs free");
        int rc = run_filter(p, ns, io->u[k], io->ubar[k], io->tau[k], plane_mean_host ? io->pm[k] : nullptr, true, s,
                            nullptr);
        if (rc) return rc;
        CKE(cudaEventRecord(io->ev_comp[k], s), "host io: computed");
        CKE(cudaStreamWaitEvent(io->s_out, io->ev_comp[k], 0), "host io: wait results");
        CKE(cudaMemcpyAsync(static_cast<char *>(ubar_host) + s0 * bb, io->ubar[k], ns * bb, cudaMemcpyDeviceToHost,
                            io->s_out), "host io: copy ubar out");
        CKE(cudaMemcpyAsync(static_cast<char *>(tau_host) + s0 * bt, io->tau[k], ns * bt, cudaMemcpyDeviceToHost,
                            io->s_out), "host io: copy tau out");
        if (plane_mean_host)
            CKE(cudaMemcpyAsync(reinterpret_cast<char *>(plane_mean_host) + s0 * bp, io->pm[k], ns * bp,
                                cudaMemcpyDeviceToHost, io->s_out), "host io: copy plane means out");
        CKE(cudaEventRecord(io->ev_out[k], io->s_out), "host io: copied out");
    }
    CKE(cudaStreamWaitEvent(s, io->ev_out[(ngroups - 1) & 1], 0), "host io: join");
#undef CKE
    return EF_OK;
}

}  // extern "C"
