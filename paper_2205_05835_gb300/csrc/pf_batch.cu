// Batched execution of many independent drops (uneven grid sizes and physical
// parameters): one context and one CUDA stream per instance, all in one
// caller-owned workspace, advanced concurrently by a pool of host threads so
// that the small, latency-bound kernels of different instances overlap on the
// GPU. Instances are handed out largest first from an atomic counter (dynamic
// load balance); each thread sleeps in blocking-sync waits instead of
// spinning. Every instance is computed exactly as by pf_step on its own.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pf.h"
#include "pf_internal.h"

struct pf_batch {
    std::vector<pf_ctx*> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<int> order;      // instances by decreasing cell count
    int nthreads = 1;
    bool graphs = false;         // every instance replays a captured step graph
    std::string err;
};

namespace {

thread_local std::string g_batch_error;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

long long cells_of(const pf_params& p) {
    long long n = 1;
    for (int d = 0; d < p.dim; ++d) n *= p.n[d];
    return n;
}

}  // namespace

extern "C" {
pf_status pf_batch_step(pf_batch* b, int nsteps);
}

extern "C" {

pf_status pf_batch_workspace_size(const pf_params* prms, int count, size_t* bytes) {
    if (!prms || count < 1 || !bytes) {
        g_batch_error = "prms and bytes must be non-NULL and count >= 1";
        return PF_ERR_INVALID;
    }
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        size_t b = 0;
        pf_status s = pf_workspace_size(&prms[i], &b);
        if (s != PF_OK) {
            g_batch_error = "instance " + std::to_string(i) + ": " + pf_last_error(nullptr);
            return s;
        }
        total += align256(b);
    }
    *bytes = total;
    return PF_OK;
}

pf_status pf_batch_init(const pf_params* prms, int count, void* workspace, size_t workspace_bytes,
                        int nthreads, pf_batch** out) {
    if (!out) return PF_ERR_INVALID;
    *out = nullptr;
    size_t need = 0;
    pf_status s = pf_batch_workspace_size(prms, count, &need);
    if (s != PF_OK) return s;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need) {
        g_batch_error = "workspace NULL, not 256-byte aligned or smaller than pf_batch_workspace_size";
        return PF_ERR_WORKSPACE;
    }
    pf_batch* b = new (std::nothrow) pf_batch();
    if (!b) return PF_ERR_INVALID;
    b->nthreads = nthreads > 0 ? nthreads : 16;
    char* base = static_cast<char*>(workspace);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        size_t bi = 0;
        pf_workspace_size(&prms[i], &bi);
        cudaStream_t st = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        pf_ctx* c = nullptr;
        if (e == cudaSuccess) s = pf_init(&prms[i], base + off, bi, nullptr, st, &c);
        if (e != cudaSuccess || s != PF_OK) {
            g_batch_error = e != cudaSuccess ? std::string("cudaStreamCreate: ") + cudaGetErrorString(e)
                                             : "instance " + std::to_string(i) + ": " +
                                                   pf_last_error(nullptr);
            if (st) cudaStreamDestroy(st);
            pf_batch_destroy(b);
            return e != cudaSuccess ? PF_ERR_CUDA : s;
        }
        pf::ctx_set_blocking(c, 1);
        b->ctx.push_back(c);
        b->streams.push_back(st);
        off += align256(bi);
    }
    b->graphs = true;
    for (int i = 0; i < count; ++i) b->graphs = b->graphs && prms[i].use_graph == 1;
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        return cells_of(prms[x]) > cells_of(prms[y]);
    });
    *out = b;
    return PF_OK;
}

// Graph mode: one host thread enqueues the step-graph replays of every
// instance on its own stream (largest first), then waits for each; the first
// steps of instances that have no graph yet run host-driven inside step_begin.
static pf_status batch_run_graphs(pf_batch* b, int nsteps, const int* each) {
    const int count = (int)b->ctx.size();
    int status = PF_OK, failed = -1;
    std::vector<char> begun(count, 0);
    for (int t = 0; t < count; ++t) {
        const int i = b->order[t];
        const int k = each ? each[i] : nsteps;
        if (k <= 0) continue;
        const int s = pf::ctx_step_begin(b->ctx[i], k);
        begun[i] = 1;
        if (s != PF_OK && status == PF_OK) { status = s; failed = i; }
    }
    for (int t = 0; t < count; ++t) {
        const int i = b->order[t];
        if (!begun[i]) continue;
        const int s = pf::ctx_step_end(b->ctx[i]);
        if (s != PF_OK && status == PF_OK) { status = s; failed = i; }
    }
    if (status != PF_OK) {
        b->err = "instance " + std::to_string(failed) + ": " + pf_last_error(b->ctx[failed]);
        return (pf_status)status;
    }
    b->err.clear();
    return PF_OK;
}

static pf_status batch_run(pf_batch* b, int nsteps, const int* each) {
    if (b->graphs) return batch_run_graphs(b, nsteps, each);
    const int count = (int)b->ctx.size();
    std::atomic<int> next(0);
    std::atomic<int> status((int)PF_OK);
    std::atomic<int> failed(-1);
    int dev = 0;
    cudaGetDevice(&dev);
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            const int t = next.fetch_add(1);
            if (t >= count) break;
            const int i = b->order[t];
            const int k = each ? each[i] : nsteps;
            if (k <= 0) continue;
            pf_status s = pf_step(b->ctx[i], k);
            if (s != PF_OK) {
                int expect = (int)PF_OK;
                if (status.compare_exchange_strong(expect, (int)s)) failed.store(i);
            }
        }
    };
    const int nt = std::min(b->nthreads, count);
    std::vector<std::thread> pool;
    pool.reserve(nt);
    for (int k = 0; k < nt; ++k) pool.emplace_back(worker);
    for (auto& th : pool) th.join();
    if (status.load() != PF_OK) {
        const int i = failed.load();
        b->err = "instance " + std::to_string(i) + ": " + pf_last_error(b->ctx[i]);
        return (pf_status)status.load();
    }
    b->err.clear();
    return PF_OK;
}

pf_status pf_batch_step(pf_batch* b, int nsteps) {
    if (!b || nsteps < 0) return PF_ERR_INVALID;
    return batch_run(b, nsteps, nullptr);
}

pf_status pf_batch_step_each(pf_batch* b, const int* nsteps) {
    if (!b || !nsteps) return PF_ERR_INVALID;
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (nsteps[i] < 0) return PF_ERR_INVALID;
    return batch_run(b, 0, nsteps);
}

int pf_batch_size(const pf_batch* b) { return b ? (int)b->ctx.size() : 0; }

pf_ctx* pf_batch_context(pf_batch* b, int i) {
    if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
    return b->ctx[i];
}

void pf_batch_destroy(pf_batch* b) {
    if (!b) return;
    for (pf_ctx* c : b->ctx) pf_destroy(c);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    delete b;
}

const char* pf_batch_last_error(const pf_batch* b) {
    return b ? b->err.c_str() : g_batch_error.c_str();
}

}  // extern "C"
