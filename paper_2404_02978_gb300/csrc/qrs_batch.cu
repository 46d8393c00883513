// qrs_batch.cu -- host side of the batched piston launch (many interferometers
// of uneven aperture count, N_f and realisation count in one persistent
// kernel), its CUDA-graph cache and the kernel-shape autotuner.
//
// Persistent launch: the jobs are sorted by descending cost per item
// (N_f (n_ap + 8): the per-(aperture, term) filter and sum plus the per-term
// draw), their realisations numbered in that order (item_begin prefix sums),
// the descriptor table uploaded from pinned staging, the queue counter
// zeroed, and one persistent grid drains the queue.
//
// Graph cache: with QRS_PISTON_GRAPH, the exact job set (descriptor bytes,
// which include the caller's device pointers) keys a captured graph of
// {counter reset, persistent kernel} whose descriptor table lives in a device
// buffer owned by the cache entry; a repeated job set replays the graph.
// Up to kGraphCache entries, least recently used evicted.
//
// Autotuner: for each job-set shape (log2 buckets of the job count, item
// count, mean N_f and mean aperture count) every persistent kernel shape is
// timed twice on the real job set and the fastest kept, in memory and, if the
// environment names a file in QRS_AUTOTUNE_CACHE, in that file (lines
// "<bucket> <shape>").  The first call for a new shape synchronises its
// stream while it times the candidates.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "qrs_internal.h"
#include "qrs_piston.h"

namespace qrs {

namespace {

constexpr int kGraphCache = 8;

struct GraphEntry {
    uint64_t key = 0;
    std::vector<unsigned char> bytes;  // exact descriptor table (collision check)
    void* d_buf = nullptr;             // descriptor table + queue counter
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
};

struct PistonState {
    cudaEvent_t stage_ev = nullptr;
    bool stage_pending = false;
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;
    std::map<std::string, int> tuned;
    bool file_loaded = false;
    uint64_t tick = 0;
};

PistonState* state(qrs_handle* h)
{
    if (!h->piston_state) h->piston_state = new PistonState();
    return static_cast<PistonState*>(h->piston_state);
}

uint64_t fnv1a(const unsigned char* p, size_t n)
{
    uint64_t x = 1469598103934665603ULL;
    for (size_t i = 0; i < n; ++i) {
        x ^= p[i];
        x *= 1099511628211ULL;
    }
    return x;
}

int ilog2_bucket(double v) { return v <= 1.0 ? 0 : (int)std::floor(std::log2(v)); }

std::string bucket_of(const std::vector<PistonJobDev>& jobs, int64_t n_items)
{
    double nf = 0.0, nap = 0.0;
    for (const PistonJobDev& J : jobs) {
        nf += (double)J.p.n_f * (double)J.n_real;
        nap += (double)J.n_ap * (double)J.n_real;
    }
    nf /= (double)std::max<int64_t>(n_items, 1);
    nap /= (double)std::max<int64_t>(n_items, 1);
    char buf[128];
    snprintf(buf, sizeof(buf), "piston:jobs%d:items%d:nf%d:nap%d", ilog2_bucket((double)jobs.size()),
             ilog2_bucket((double)n_items), ilog2_bucket(nf), ilog2_bucket(nap));
    return buf;
}

void load_tune_file(PistonState* st)
{
    st->file_loaded = true;
    const char* path = getenv("QRS_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[256];
    int shape;
    while (fscanf(f, "%255s %d", key, &shape) == 2)
        if (shape >= 0 && shape < piston_shape_count()) st->tuned[key] = shape;
    fclose(f);
}

void save_tune(const std::string& key, int shape)
{
    const char* path = getenv("QRS_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", key.c_str(), shape);
    fclose(f);
}

// Time every kernel shape on the uploaded job table (twice) and keep the fastest.
qrs_status autotune(qrs_handle* h, const std::vector<PistonJobDev>& jobs, int64_t n_items, const PistonJobDev* d_jobs,
                    unsigned long long* d_counter, cudaStream_t s, int* shape_out)
{
    PistonState* st = state(h);
    if (!st->file_loaded) load_tune_file(st);
    const std::string key = bucket_of(jobs, n_items);
    auto it = st->tuned.find(key);
    if (it != st->tuned.end()) {
        *shape_out = it->second;
        return QRS_OK;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(h, QRS_ERR_CUDA, "autotune event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(h, QRS_ERR_CUDA, "autotune event");
    }
    int best = 0;
    float best_ms = 1e30f;
    // two rounds over the shapes, the faster of each shape's two timings: the
    // first launch of a kernel also pays for its code and the job tables
    // reaching the caches, which would favour whichever shape runs later
    for (int k = 0; k < 2 * piston_shape_count(); ++k) {
        const int shape = k % piston_shape_count();
        cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess)
            e = launch_piston_persistent(shape, d_jobs, (int)jobs.size(), n_items, d_counter, h->num_sms, h->d_err, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(h, e, "autotune launch");
        }
        ++h->launches;
        if (ms < best_ms) {
            best_ms = ms;
            best = shape;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st->tuned[key] = best;
    save_tune(key, best);
    *shape_out = best;
    return QRS_OK;
}

}  // namespace

void destroy_piston_state(qrs_handle* h)
{
    PistonState* st = static_cast<PistonState*>(h->piston_state);
    if (!st) return;
    for (GraphEntry& g : st->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        if (g.d_buf) cudaFree(g.d_buf);
    }
    if (st->stage_ev) cudaEventDestroy(st->stage_ev);
    if (st->cap_stream) cudaStreamDestroy(st->cap_stream);
    delete st;
    h->piston_state = nullptr;
}

// jobs: validated descriptors (item_begin unset).  Sorts them, then runs the
// persistent kernel directly or through the graph cache.
qrs_status run_piston_batch(qrs_handle* h, std::vector<PistonJobDev>& jobs, bool graph, cudaStream_t s)
{
    std::vector<PistonJobDev> js;
    js.reserve(jobs.size());
    for (const PistonJobDev& J : jobs)
        if (J.n_real > 0) js.push_back(J);
    if (js.empty()) return QRS_OK;
    std::stable_sort(js.begin(), js.end(), [](const PistonJobDev& a, const PistonJobDev& b) {
        return (double)a.p.n_f * (a.n_ap + 8) > (double)b.p.n_f * (b.n_ap + 8);
    });
    int64_t n_items = 0;
    for (PistonJobDev& J : js) {
        J.item_begin = n_items;
        n_items += J.n_real;
    }
    const size_t table = js.size() * sizeof(PistonJobDev);
    const size_t counter_off = (table + 255) & ~(size_t)255;
    const size_t bytes = counter_off + 256;
    PistonState* st = state(h);
    cudaError_t e;

    if (!graph) {
        qrs_status q = ensure_work(h, bytes);
        if (q != QRS_OK) return q;
        if (!st->stage_ev && (e = cudaEventCreateWithFlags(&st->stage_ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(h, e, "staging event");
        if (h->stage_bytes < table) {
            if (h->h_stage) {
                if (st->stage_pending) cudaEventSynchronize(st->stage_ev);
                cudaFreeHost(h->h_stage);
                h->h_stage = nullptr;
                h->stage_bytes = 0;
            }
            if ((e = cudaMallocHost(&h->h_stage, std::max(table, (size_t)1 << 16))) != cudaSuccess)
                return cuda_fail(h, e, "pinned staging");
            h->stage_bytes = std::max(table, (size_t)1 << 16);
        } else if (st->stage_pending) {
            cudaEventSynchronize(st->stage_ev);  // the previous upload has left the staging buffer
        }
        std::memcpy(h->h_stage, js.data(), table);
        unsigned char* base = static_cast<unsigned char*>(h->d_work);
        auto* d_jobs = reinterpret_cast<PistonJobDev*>(base);
        auto* d_counter = reinterpret_cast<unsigned long long*>(base + counter_off);
        if ((e = cudaMemcpyAsync(d_jobs, h->h_stage, table, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(h, e, "descriptor upload");
        if ((e = cudaEventRecord(st->stage_ev, s)) != cudaSuccess) return cuda_fail(h, e, "staging event");
        st->stage_pending = true;
        int shape = 0;
        qrs_status q2 = autotune(h, js, n_items, d_jobs, d_counter, s, &shape);
        if (q2 != QRS_OK) return q2;
        if ((e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), s)) != cudaSuccess)
            return cuda_fail(h, e, "queue reset");
        e = launch_piston_persistent(shape, d_jobs, (int)js.size(), n_items, d_counter, h->num_sms, h->d_err, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "persistent piston launch");
        ++h->launches;
        return QRS_OK;
    }

    // ---- graph path
    const unsigned char* raw = reinterpret_cast<const unsigned char*>(js.data());
    const uint64_t key = fnv1a(raw, table) ^ (uint64_t)n_items;
    ++st->tick;
    for (GraphEntry& g : st->graphs) {
        if (g.key == key && g.bytes.size() == table && std::memcmp(g.bytes.data(), raw, table) == 0) {
            g.last_use = st->tick;
            if ((e = cudaGraphLaunch(g.exec, s)) != cudaSuccess) return cuda_fail(h, e, "graph launch");
            ++h->launches;
            return QRS_OK;
        }
    }
    if (!st->cap_stream && (e = cudaStreamCreateWithFlags(&st->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(h, e, "capture stream");
    if ((int)st->graphs.size() >= kGraphCache) {  // evict the least recently used entry
        auto lru = std::min_element(st->graphs.begin(), st->graphs.end(),
                                    [](const GraphEntry& a, const GraphEntry& b) { return a.last_use < b.last_use; });
        cudaDeviceSynchronize();  // a replay of it may still be queued
        cudaGraphExecDestroy(lru->exec);
        cudaGraphDestroy(lru->graph);
        cudaFree(lru->d_buf);
        st->graphs.erase(lru);
    }
    GraphEntry g;
    g.key = key;
    g.bytes.assign(raw, raw + table);
    if ((e = cudaMalloc(&g.d_buf, bytes)) != cudaSuccess) return cuda_fail(h, e, "graph descriptor buffer");
    auto* d_jobs = reinterpret_cast<PistonJobDev*>(g.d_buf);
    auto* d_counter = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(g.d_buf) + counter_off);
    e = cudaMemcpy(d_jobs, raw, table, cudaMemcpyHostToDevice);
    int shape = 0;
    qrs_status q = QRS_OK;
    if (e == cudaSuccess) q = autotune(h, js, n_items, d_jobs, d_counter, st->cap_stream, &shape);
    if (e != cudaSuccess || q != QRS_OK) {
        cudaFree(g.d_buf);
        return e != cudaSuccess ? cuda_fail(h, e, "graph descriptor upload") : q;
    }
    e = cudaStreamBeginCapture(st->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), st->cap_stream);
        if (e1 == cudaSuccess)
            e1 = launch_piston_persistent(shape, d_jobs, (int)js.size(), n_items, d_counter, h->num_sms, h->d_err,
                                          st->cap_stream);
        e = cudaStreamEndCapture(st->cap_stream, &g.graph);
        if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (e != cudaSuccess) {
        if (g.graph) cudaGraphDestroy(g.graph);
        cudaFree(g.d_buf);
        return cuda_fail(h, e, "graph capture");
    }
    g.last_use = st->tick;
    st->graphs.push_back(std::move(g));
    if ((e = cudaGraphLaunch(st->graphs.back().exec, s)) != cudaSuccess) return cuda_fail(h, e, "graph launch");
    ++h->launches;
    return QRS_OK;
}

}  // namespace qrs
