// Many independent cross-validation problems of uneven size in one call
// (pichol_batch_*).  Each problem keeps its own context, laid out inside one
// workspace.  pichol_batch_run forks from the caller's stream onto the batch's
// internal streams (problems assigned longest first, round-robin), runs every
// problem's whole pipeline (Gram blocks, sampled factors, fit, interpolated
// hold-out scores) on its stream, and joins back; the fork and join are event
// waits, so the whole batch can be captured into one CUDA graph and replayed.
#include "internal.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

struct pichol_batch {
    int nprob;
    int nstreams;
    std::vector<pichol_ctx*> ctx;
    std::vector<size_t> off;        // workspace offset of each problem
    std::vector<int> order;         // problems, most expensive first
    size_t need_bytes;
    char* ws;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev;    // fork + one join event per stream
    bool have_streams;
};

namespace {

double cost_of(const pichol_config& c)
{
    // factorisations dominate: k g d^3 / 3, then the solves k q d^2 c
    const double d = (double)c.d;
    return c.k * (c.g * d * d * d / 3.0 + 4.0 * c.q * d * d * (double)c.c);
}

void free_streams(pichol_batch* b)
{
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    b->streams.clear();
    b->ev.clear();
    b->have_streams = false;
}

pichol_status make_streams(pichol_batch* b)
{
    if (b->have_streams && (int)b->streams.size() == b->nstreams) return PICHOL_OK;
    free_streams(b);
    for (int i = 0; i < b->nstreams; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return PICHOL_ERR_CUDA;
        b->streams.push_back(s);
    }
    for (int i = 0; i < b->nstreams + 1; ++i) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PICHOL_ERR_CUDA;
        b->ev.push_back(e);
    }
    b->have_streams = true;
    return PICHOL_OK;
}

}  // namespace

extern "C" {

pichol_status pichol_batch_create(const pichol_config* cfgs, int32_t nprob, int32_t nstreams, pichol_batch** out)
{
    if (out) *out = nullptr;
    if (!cfgs || !out || nprob < 1 || nprob > 4096 || nstreams < 1 || nstreams > 64) return PICHOL_ERR_INVALID_ARG;
    pichol_batch* b = new (std::nothrow) pichol_batch();
    if (!b) return PICHOL_ERR_INVALID_ARG;
    b->nprob = nprob;
    b->nstreams = nstreams;
    b->ws = nullptr;
    b->have_streams = false;
    size_t off = 0;
    for (int i = 0; i < nprob; ++i) {
        pichol_ctx* c = nullptr;
        pichol_status st = pichol_create(&cfgs[i], &c);
        if (st != PICHOL_OK) {
            for (pichol_ctx* x : b->ctx) pichol_destroy(x);
            delete b;
            return st;
        }
        c->tune.diag_exclusive = 0;   // other problems' work fills the SMs instead
        b->ctx.push_back(c);
        b->off.push_back(off);
        size_t need = 0;
        pichol_workspace_size(c, &need);
        off += (need + 255) & ~size_t(255);
    }
    b->need_bytes = off;
    b->order.resize(nprob);
    for (int i = 0; i < nprob; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return cost_of(cfgs[x]) > cost_of(cfgs[y]); });
    *out = b;
    return PICHOL_OK;
}

pichol_status pichol_batch_workspace_size(const pichol_batch* b, size_t* bytes)
{
    if (!b || !bytes) return PICHOL_ERR_INVALID_ARG;
    *bytes = b->need_bytes;
    return PICHOL_OK;
}

pichol_status pichol_batch_set_workspace(pichol_batch* b, void* workspace, size_t bytes)
{
    if (!b || !workspace) return PICHOL_ERR_INVALID_ARG;
    if (bytes < b->need_bytes || ((uintptr_t)workspace & 255u)) return PICHOL_ERR_WORKSPACE;
    b->ws = nullptr;                      // until every problem has its part
    for (int i = 0; i < b->nprob; ++i) {
        size_t need = 0;
        pichol_workspace_size(b->ctx[i], &need);
        pichol_status st = pichol_set_workspace(b->ctx[i], (char*)workspace + b->off[i], need);
        if (st != PICHOL_OK) return st;
    }
    b->ws = (char*)workspace;
    return PICHOL_OK;
}

pichol_status pichol_batch_set_streams(pichol_batch* b, int32_t nstreams)
{
    if (!b || nstreams < 1 || nstreams > 64) return PICHOL_ERR_INVALID_ARG;
    if (nstreams != b->nstreams) {
        free_streams(b);
        b->nstreams = nstreams;
    }
    return PICHOL_OK;
}

pichol_status pichol_batch_set_tuning(pichol_batch* b, const pichol_tuning* t)
{
    if (!b || !t || b->ctx.empty()) return PICHOL_ERR_INVALID_ARG;
    pichol_status st = pichol_set_tuning(b->ctx[0], t);   // validates; changes nothing on error
    if (st != PICHOL_OK) return st;
    for (pichol_ctx* c : b->ctx) c->tune = *t;
    return PICHOL_OK;
}

pichol_status pichol_batch_run(pichol_batch* b, const void* const* X, const void* const* Y, double* const* E_out,
                               int32_t* t_star, void* stream)
{
    pichol::CallRange range_(__func__);
    if (!b || !X || !Y || !E_out || !t_star) return PICHOL_ERR_INVALID_ARG;
    if (!b->ws) return PICHOL_ERR_WORKSPACE;
    for (int i = 0; i < b->nprob; ++i)
        if (!X[i] || !Y[i] || !E_out[i]) return PICHOL_ERR_INVALID_ARG;
    pichol_status st = make_streams(b);
    if (st != PICHOL_OK) return st;
    cudaStream_t origin = (cudaStream_t)stream;
    // fork: every internal stream waits for the work already on the caller's stream
    if (cudaEventRecord(b->ev[0], origin) != cudaSuccess) return PICHOL_ERR_CUDA;
    for (int s = 0; s < b->nstreams; ++s)
        if (cudaStreamWaitEvent(b->streams[s], b->ev[0], 0) != cudaSuccess) return PICHOL_ERR_CUDA;
    // after the first failing call no further problem is enqueued, but the join
    // below still runs, so the caller's stream stays ordered after what was
    // enqueued and a capture is never left with unjoined streams
    for (int r = 0; r < b->nprob && st == PICHOL_OK; ++r) {
        const int i = b->order[r];
        cudaStream_t s = b->streams[r % b->nstreams];
        pichol_ctx* c = b->ctx[i];
        if ((st = pichol_hessian(c, X[i], Y[i], nullptr, s)) != PICHOL_OK) break;
        if ((st = pichol_factor_samples(c, nullptr, s)) != PICHOL_OK) break;
        if ((st = pichol_fit(c, nullptr, s)) != PICHOL_OK) break;
        st = pichol_eval_holdout(c, nullptr, E_out[i], t_star + i, nullptr, s);
    }
    // join: the caller's stream waits for every internal stream
    for (int s = 0; s < b->nstreams; ++s) {
        if (cudaEventRecord(b->ev[1 + s], b->streams[s]) != cudaSuccess ||
            cudaStreamWaitEvent(origin, b->ev[1 + s], 0) != cudaSuccess)
            return st != PICHOL_OK ? st : PICHOL_ERR_CUDA;
    }
    return st;
}

pichol_status pichol_batch_get_info(pichol_batch* b, int32_t i, pichol_info* info, void* stream)
{
    if (!b || i < 0 || i >= b->nprob) return PICHOL_ERR_INVALID_ARG;
    return pichol_get_info(b->ctx[i], info, stream);
}

pichol_status pichol_batch_set_timing(pichol_batch* b, int32_t max_launches)
{
    if (!b) return PICHOL_ERR_INVALID_ARG;
    for (pichol_ctx* c : b->ctx) {
        pichol_status st = pichol_set_timing(c, max_launches);
        if (st != PICHOL_OK) return st;
    }
    return PICHOL_OK;
}

pichol_status pichol_batch_stage_times(pichol_batch* b, int32_t i, double* ms, int64_t* launches, int32_t n_stages,
                                       void* stream)
{
    if (!b || i < 0 || i >= b->nprob) return PICHOL_ERR_INVALID_ARG;
    return pichol_stage_times(b->ctx[i], ms, launches, n_stages, stream);
}

int64_t pichol_batch_launch_count(const pichol_batch* b)
{
    if (!b) return 0;
    int64_t n = 0;
    for (pichol_ctx* c : b->ctx) n += pichol_launch_count(c);
    return n;
}

void pichol_batch_destroy(pichol_batch* b)
{
    if (!b) return;
    free_streams(b);
    for (pichol_ctx* c : b->ctx) pichol_destroy(c);
    delete b;
}

}  // extern "C"
