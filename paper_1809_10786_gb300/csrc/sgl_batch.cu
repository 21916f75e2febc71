// sgl_batch.cu -- many independent transforms (each its own B, points and coefficients)
// issued together (the definition of the NDSGLFT applied per instance).  One plan per instance;
// the instances are spread over L lanes, each a stream of its own with its own FFT work buffers
// (shared by the plans of that lane, sized for the largest of them), so that the small kernels
// of different instances run side by side on the GPU.  Instances go to lanes by a cost estimate
// (longest first onto the least loaded lane).  A batch call forks from the batch's stream into the
// lanes and joins back; it can be captured into one CUDA graph (fork and join included) and
// replayed while the pointers and point counts match.  sgl_batch_autotune times the call for
// several lane counts and keeps the fastest, cached in a JSON file.
#include "sgl_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <new>
#include <sstream>
#include <string>
#include <vector>

struct sgl_batch {
    int n = 0;
    cudaStream_t stream = nullptr;
    std::vector<sgl_plan *> plans;
    int precision = 0, window = 0, q = 0;
    double sigma = 0.0;
    std::vector<int> Bs;
    std::vector<int64_t> Mmax;
    // lanes: a stream, FFT work buffers and the instances (in issue order) of each
    int lanes = 0;
    std::vector<cudaStream_t> lane_stream;
    std::vector<void *> lane_bufA, lane_bufB;
    std::vector<size_t> lane_bytesA, lane_bytesB;
    std::vector<std::vector<int>> lane_items;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    bool use_graph = false;
    // one cached graph per call kind (0 forward, 1 adjoint), keyed on pointers and sizes
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::vector<uintptr_t> key[2];
    int64_t graph_launches = 0;
    // graphs are captured and replayed on a private stream (the legacy default stream
    // cannot be captured), ordered after and before the caller's stream by events
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {

constexpr int kMaxLanes = 32;

void free_lanes(sgl_batch *b) {
    for (cudaStream_t s : b->lane_stream)
        if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    for (void *p : b->lane_bufA) cudaFree(p);
    for (void *p : b->lane_bufB) cudaFree(p);
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    b->lane_stream.clear();
    b->lane_bufA.clear();
    b->lane_bufB.clear();
    b->lane_bytesA.clear();
    b->lane_bytesB.clear();
    b->ev_join.clear();
    b->lane_items.clear();
    b->lanes = 0;
}

void drop_graphs(sgl_batch *b) {
    for (int k = 0; k < 2; ++k) {
        if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
        b->exec[k] = nullptr;
        b->key[k].clear();
    }
}

sgl_status fail_batch(sgl_batch *b, sgl_status st, const std::string &msg) {
    if (b) {
        for (sgl_plan *p : b->plans) sgl_plan_destroy(p);
        drop_graphs(b);
        free_lanes(b);
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        if (b->ev_in) cudaEventDestroy(b->ev_in);
        if (b->ev_out) cudaEventDestroy(b->ev_out);
        if (b->ev_fork) cudaEventDestroy(b->ev_fork);
        delete b;
    }
    return sgl::set_error(st, msg);
}

// Cost estimate of one forward + adjoint of an instance (milliseconds, GB300 scale): the
// conversions (O(B^4) FP64), the FFT passes per stored grid cell and the windowed loops per tap.
double instance_cost(int B, int64_t M, int precision, int q, double sigma) {
    size_t a = 0, c = 0;
    sgl::plan_work_sizes(B, precision, q, sigma, &a, &c);
    const double cell_bytes = precision == SGL_FP32_MIXED ? 8.0 : 16.0;
    const double cells = (double)a / cell_bytes;
    const double tap = precision == SGL_FP32_MIXED ? 5.8e-10 : 6.2e-9;
    const double cell = precision == SGL_FP32_MIXED ? 6.8e-8 : 3.8e-7;
    const double conv = 1.4e-8;                    // about 0.75 ms at B = 64 for both directions
    return (double)M * 8.0 * q * q * q * tap + cells * cell + conv * std::pow((double)B, 4.0) + 0.02;
}

}  // namespace

namespace {

struct Lanes {
    std::vector<cudaStream_t> stream;
    std::vector<void *> bufA, bufB;
    std::vector<size_t> bytesA, bytesB;
    std::vector<cudaEvent_t> join;
    std::vector<std::vector<int>> items;
};

void free_lane_set(Lanes &x) {
    for (cudaStream_t s : x.stream)
        if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    for (void *p : x.bufA) cudaFree(p);
    for (void *p : x.bufB) cudaFree(p);
    for (cudaEvent_t e : x.join)
        if (e) cudaEventDestroy(e);
    x = Lanes{};
}

// Spread the instances over L lanes (longest estimated first, onto the least loaded lane), make
// each lane's stream, join event and work buffers, then (only if all of that succeeded) release
// the previous lanes and point the instances' plans, if they exist yet, at their new lane.
cudaError_t assign_lanes(sgl_batch *b, int L) {
    std::vector<std::pair<double, int>> order(b->n);
    for (int i = 0; i < b->n; ++i) order[i] = {instance_cost(b->Bs[i], b->Mmax[i], b->precision, b->q, b->sigma), i};
    std::stable_sort(order.begin(), order.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    std::vector<double> load(L, 0.0);
    Lanes nl;
    nl.items.assign(L, {});
    for (const auto &o : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += o.first;
        nl.items[l].push_back(o.second);
    }
    for (auto &v : nl.items) std::sort(v.begin(), v.end());     // issue order within a lane: instance order
    nl.stream.assign(L, nullptr);
    nl.bufA.assign(L, nullptr);
    nl.bufB.assign(L, nullptr);
    nl.bytesA.assign(L, 0);
    nl.bytesB.assign(L, 0);
    nl.join.assign(L, nullptr);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        for (int i : nl.items[l]) {
            size_t a = 0, c = 0;
            sgl::plan_work_sizes(b->Bs[i], b->precision, b->q, b->sigma, &a, &c);
            nl.bytesA[l] = std::max(nl.bytesA[l], a);
            nl.bytesB[l] = std::max(nl.bytesB[l], c);
        }
        e = cudaStreamCreateWithFlags(&nl.stream[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&nl.join[l], cudaEventDisableTiming);
        if (e == cudaSuccess && nl.bytesA[l]) e = sgl::device_malloc(&nl.bufA[l], nl.bytesA[l]);
        if (e == cudaSuccess && nl.bytesB[l]) e = sgl::device_malloc(&nl.bufB[l], nl.bytesB[l]);
    }
    if (e != cudaSuccess) {
        free_lane_set(nl);
        return e;
    }
    drop_graphs(b);
    free_lanes(b);                                   // waits for the old lanes' work first
    b->lanes = L;
    b->lane_stream = nl.stream;
    b->lane_bufA = nl.bufA;
    b->lane_bufB = nl.bufB;
    b->lane_bytesA = nl.bytesA;
    b->lane_bytesB = nl.bytesB;
    b->ev_join = nl.join;
    b->lane_items = nl.items;
    if (!b->plans.empty())
        for (int l = 0; l < L; ++l)
            for (int i : nl.items[l]) {
                sgl_plan *p = b->plans[i];
                p->b.bufA = nl.bufA[l];
                p->b.bufB = nl.bufB[l];
                p->b.bufA_bytes = nl.bytesA[l];
                p->b.bufB_bytes = nl.bytesB[l];
                p->stream = nl.stream[l];
            }
    return cudaSuccess;
}

// every lane waits for the work already on stream s (fork) ...
cudaError_t fork(sgl_batch *b, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(b->ev_fork, s);
    for (int l = 0; l < b->lanes && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(b->lane_stream[l], b->ev_fork, 0);
    return e;
}

// ... and stream s waits for every lane (join)
cudaError_t join(sgl_batch *b, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < b->lanes && e == cudaSuccess; ++l) {
        e = cudaEventRecord(b->ev_join[l], b->lane_stream[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join[l], 0);
    }
    return e;
}

std::vector<uintptr_t> make_key(const sgl_batch *b, const void *const *in, const void *const *out) {
    std::vector<uintptr_t> k;
    k.reserve(3 * b->n);
    for (int i = 0; i < b->n; ++i) {
        k.push_back((uintptr_t)in[i]);
        k.push_back((uintptr_t)out[i]);
        k.push_back((uintptr_t)b->plans[i]->M);
    }
    return k;
}

// issue every instance's call on its lane, lane by lane (the lanes run concurrently)
sgl_status issue(sgl_batch *b, int kind, const double *const *in, double *const *out) {
    for (int l = 0; l < b->lanes; ++l)
        for (int i : b->lane_items[l]) {
            sgl_status st = kind == 0 ? sgl_forward(b->plans[i], in[i], out[i]) : sgl_adjoint(b->plans[i], in[i], out[i]);
            if (st != SGL_OK) return sgl::set_error(st, "instance " + std::to_string(i) + ": " + sgl_last_error());
        }
    return SGL_OK;
}

sgl_status cuda_err(cudaError_t e, const char *what) {
    return sgl::set_error(SGL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

sgl_status run(sgl_batch *b, int kind, const double *const *in, double *const *out) {
    if (!b) return sgl::set_error(SGL_ERR_ARG, "batch is NULL");
    if (!in || !out) return sgl::set_error(SGL_ERR_ARG, "pointer arrays must not be NULL");
    for (int i = 0; i < b->n; ++i)
        if (!b->plans[i]->points_set) return sgl::set_error(SGL_ERR_STATE, "sgl_batch_set_points has not been called");
    if (!b->use_graph) {
        cudaError_t e = fork(b, b->stream);
        if (e != cudaSuccess) return cuda_err(e, "batch fork");
        sgl_status st = issue(b, kind, in, out);
        e = join(b, b->stream);
        if (st != SGL_OK) return st;
        if (e != cudaSuccess) return cuda_err(e, "batch join");
        return sgl::set_error(SGL_OK, "");
    }
    std::vector<uintptr_t> k = make_key(b, (const void *const *)in, (const void *const *)out);
    cudaError_t e = cudaEventRecord(b->ev_in, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap_stream, b->ev_in, 0);
    if (e != cudaSuccess) return cuda_err(e, "stream ordering");
    if (!b->exec[kind] || k != b->key[kind]) {
        if (b->exec[kind]) {
            cudaGraphExecDestroy(b->exec[kind]);
            b->exec[kind] = nullptr;
        }
        // the capture follows the fork into every lane and ends with the join
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed);
        sgl_status st = SGL_OK;
        if (e == cudaSuccess) {
            e = fork(b, b->cap_stream);
            if (e == cudaSuccess) st = issue(b, kind, in, out);
            const cudaError_t ej = join(b, b->cap_stream);
            if (e == cudaSuccess) e = ej;
            const cudaError_t ee = cudaStreamEndCapture(b->cap_stream, &graph);
            if (e == cudaSuccess) e = ee;
        }
        if (st != SGL_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return st != SGL_OK ? st : cuda_err(e, "graph capture");
        }
        e = cudaGraphInstantiate(&b->exec[kind], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec[kind] = nullptr;
            return cuda_err(e, "cudaGraphInstantiate");
        }
        b->key[kind] = std::move(k);
    }
    e = cudaGraphLaunch(b->exec[kind], b->cap_stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->cap_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_out, 0);
    if (e != cudaSuccess) return cuda_err(e, "cudaGraphLaunch");
    b->graph_launches += 1;
    return sgl::set_error(SGL_OK, "");
}

}  // namespace

namespace {

// ---- tuning cache: a JSON object with one entry per line,
//   "<signature>": {"lanes": L, "ms": {"1": t1, "2": t2, ...}}
// (the signature names the precision, window, q, sigma, the instance count and a 64-bit FNV-1a
// hash of the (B, M_max) list).
std::string signature(const sgl_batch *b) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](uint64_t v) {
        for (int k = 0; k < 8; ++k) {
            h ^= (v >> (8 * k)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    for (int i = 0; i < b->n; ++i) {
        mix((uint64_t)b->Bs[i]);
        mix((uint64_t)b->Mmax[i]);
    }
    char buf[160];
    std::snprintf(buf, sizeof buf, "p%d w%d q%d s%.4f n%d h%016llx", b->precision, b->window, b->q, b->sigma, b->n,
                  (unsigned long long)h);
    return buf;
}

std::map<std::string, std::string> read_cache(const std::string &path) {
    std::map<std::string, std::string> m;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        const size_t a = line.find('"');
        if (a == std::string::npos) continue;
        const size_t b = line.find('"', a + 1);
        const size_t c = line.find('{', b == std::string::npos ? 0 : b);
        const size_t d = line.rfind('}');
        if (b == std::string::npos || c == std::string::npos || d == std::string::npos || d < c) continue;
        m[line.substr(a + 1, b - a - 1)] = line.substr(c, d - c + 1);
    }
    return m;
}

bool cache_lanes(const std::string &path, const std::string &key, int *lanes) {
    const auto m = read_cache(path);
    const auto it = m.find(key);
    if (it == m.end()) return false;
    const size_t k = it->second.find("\"lanes\":");
    if (k == std::string::npos) return false;
    const int L = std::atoi(it->second.c_str() + k + 8);
    if (L < 1 || L > kMaxLanes) return false;
    *lanes = L;
    return true;
}

bool cache_store(const std::string &path, const std::string &key, int lanes, const std::vector<std::pair<int, double>> &ms) {
    auto m = read_cache(path);
    std::ostringstream e;
    e << "{\"lanes\": " << lanes << ", \"ms\": {";
    for (size_t i = 0; i < ms.size(); ++i) e << (i ? ", " : "") << "\"" << ms[i].first << "\": " << ms[i].second;
    e << "}}";
    m[key] = e.str();
    const std::string tmp = path + ".tmp";
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) return false;
        f << "{\n";
        size_t i = 0;
        for (const auto &kv : m) f << "\"" << kv.first << "\": " << kv.second << (++i < m.size() ? ",\n" : "\n");
        f << "}\n";
        if (!f) return false;
    }
    return std::rename(tmp.c_str(), path.c_str()) == 0;
}

}  // namespace

extern "C" {

sgl_status sgl_batch_create(sgl_batch **out, int n, const int *B, const int64_t *M_max, int precision, int window, int q,
                            double sigma, unsigned flags, void *cuda_stream) {
    if (!out) return sgl::set_error(SGL_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 65536) return sgl::set_error(SGL_ERR_ARG, "n must be in [1, 65536]");
    if (!B || !M_max) return sgl::set_error(SGL_ERR_ARG, "B and M_max arrays must not be NULL");
    if (flags & SGL_FLAG_PROFILE) return sgl::set_error(SGL_ERR_ARG, "batches do not take SGL_FLAG_PROFILE");
    if (flags & SGL_FLAG_OVERLAP_POINTS) return sgl::set_error(SGL_ERR_ARG, "batches do not take SGL_FLAG_OVERLAP_POINTS");
    sgl_batch *b = new (std::nothrow) sgl_batch();
    if (!b) return sgl::set_error(SGL_ERR_ALLOC, "host allocation failed");
    b->n = n;
    b->stream = (cudaStream_t)cuda_stream;
    b->precision = precision;
    b->window = window;
    b->q = q;
    b->sigma = sigma;
    b->Bs.assign(B, B + n);
    b->Mmax.assign(M_max, M_max + n);
    for (int i = 0; i < n; ++i) {
        size_t a = 0, c = 0;
        if (sgl::plan_work_sizes(B[i], precision, q, sigma, &a, &c) != SGL_OK || M_max[i] < 0)
            return fail_batch(b, SGL_ERR_ARG, "instance " + std::to_string(i) + ": invalid B, M_max, q or sigma");
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail_batch(b, SGL_ERR_CUDA, std::string("batch streams: ") + cudaGetErrorString(e));
    if ((e = assign_lanes(b, std::min(n, 8))) != cudaSuccess)
        return fail_batch(b, SGL_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    std::vector<int> lane_of(n, 0);
    for (int l = 0; l < b->lanes; ++l)
        for (int i : b->lane_items[l]) lane_of[i] = l;
    b->plans.reserve(n);
    for (int i = 0; i < n; ++i) {
        const int l = lane_of[i];
        sgl::SharedWork sw{b->lane_bufA[l], b->lane_bufB[l], b->lane_bytesA[l], b->lane_bytesB[l]};
        sgl_plan *p = nullptr;
        sgl_status st = sgl::plan_create_impl(&p, B[i], M_max[i], precision, window, q, sigma, flags, b->lane_stream[l], &sw);
        if (st != SGL_OK) return fail_batch(b, st, "instance " + std::to_string(i) + ": " + sgl_last_error());
        b->plans.push_back(p);
    }
    *out = b;
    return sgl::set_error(SGL_OK, "");
}

void sgl_batch_destroy(sgl_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (sgl_plan *p : b->plans) sgl_plan_destroy(p);
    drop_graphs(b);
    cudaStreamSynchronize(b->cap_stream);
    free_lanes(b);
    cudaStreamDestroy(b->cap_stream);
    cudaEventDestroy(b->ev_in);
    cudaEventDestroy(b->ev_out);
    cudaEventDestroy(b->ev_fork);
    delete b;
}

sgl_status sgl_batch_use_graph(sgl_batch *b, int enable) {
    if (!b) return sgl::set_error(SGL_ERR_ARG, "batch is NULL");
    b->use_graph = enable != 0;
    return sgl::set_error(SGL_OK, "");
}

sgl_status sgl_batch_set_lanes(sgl_batch *b, int lanes) {
    if (!b) return sgl::set_error(SGL_ERR_ARG, "batch is NULL");
    if (lanes < 1 || lanes > std::min(b->n, kMaxLanes))
        return sgl::set_error(SGL_ERR_ARG, "lanes must be in [1, min(n, " + std::to_string(kMaxLanes) + ")]");
    if (lanes == b->lanes) return sgl::set_error(SGL_OK, "");
    cudaStreamSynchronize(b->stream);
    const cudaError_t e = assign_lanes(b, lanes);
    if (e != cudaSuccess) return sgl::set_error(SGL_ERR_ALLOC, std::string("lane work buffers: ") + cudaGetErrorString(e));
    return sgl::set_error(SGL_OK, "");
}

sgl_status sgl_batch_lanes(const sgl_batch *b, int *lanes) {
    if (!b || !lanes) return sgl::set_error(SGL_ERR_ARG, "batch and lanes must be non-NULL");
    *lanes = b->lanes;
    return sgl::set_error(SGL_OK, "");
}

sgl_status sgl_batch_set_points(sgl_batch *b, const double *const *xyz_dev, const int64_t *M) {
    if (!b) return sgl::set_error(SGL_ERR_ARG, "batch is NULL");
    if (!xyz_dev || !M) return sgl::set_error(SGL_ERR_ARG, "pointer arrays must not be NULL");
    cudaError_t e = fork(b, b->stream);
    if (e != cudaSuccess) return cuda_err(e, "batch fork");
    sgl_status st = SGL_OK;
    for (int i = 0; i < b->n && st == SGL_OK; ++i) {
        st = sgl_set_points(b->plans[i], xyz_dev[i], M[i]);
        if (st != SGL_OK) st = sgl::set_error(st, "instance " + std::to_string(i) + ": " + sgl_last_error());
    }
    e = join(b, b->stream);
    if (st != SGL_OK) return st;
    if (e != cudaSuccess) return cuda_err(e, "batch join");
    drop_graphs(b);                                  // point counts may have changed
    return sgl::set_error(SGL_OK, "");
}

sgl_status sgl_batch_forward(sgl_batch *b, const double *const *coef_dev, double *const *vals_dev) {
    return run(b, 0, coef_dev, vals_dev);
}

sgl_status sgl_batch_adjoint(sgl_batch *b, const double *const *vals_dev, double *const *coef_dev) {
    return run(b, 1, vals_dev, coef_dev);
}

sgl_status sgl_batch_info(const sgl_batch *b, int *n, int64_t *graph_launches, int64_t *workspace_bytes) {
    if (!b) return sgl::set_error(SGL_ERR_ARG, "batch is NULL");
    if (n) *n = b->n;
    if (graph_launches) *graph_launches = b->graph_launches;
    if (workspace_bytes) {
        int64_t tot = 0;
        for (int l = 0; l < b->lanes; ++l) tot += (int64_t)(b->lane_bytesA[l] + b->lane_bytesB[l]);
        for (const sgl_plan *p : b->plans) tot += p->work_bytes;
        *workspace_bytes = tot;
    }
    return sgl::set_error(SGL_OK, "");
}

sgl_status sgl_batch_sync(sgl_batch *b) {
    if (!b) return sgl::set_error(SGL_ERR_ARG, "batch is NULL");
    for (sgl_plan *p : b->plans) {
        sgl_status st = sgl_sync(p);
        if (st != SGL_OK) return st;
    }
    if (cudaError_t e = cudaStreamSynchronize(b->stream)) return cuda_err(e, "batch stream");
    return sgl::set_error(SGL_OK, "");
}

sgl_status sgl_batch_autotune(sgl_batch *b, const char *cache_path, int *lanes_out, double *ms_out) {
    if (!b) return sgl::set_error(SGL_ERR_ARG, "batch is NULL");
    const std::string key = signature(b);
    int L = 0;
    if (cache_path && cache_lanes(cache_path, key, &L) && L <= std::min(b->n, kMaxLanes)) {
        if (sgl_status st = sgl_batch_set_lanes(b, L)) return st;
        if (lanes_out) *lanes_out = L;
        if (ms_out) *ms_out = -1.0;
        return sgl::set_error(SGL_OK, "");
    }
    for (int i = 0; i < b->n; ++i)
        if (!b->plans[i]->points_set) return sgl::set_error(SGL_ERR_STATE, "sgl_batch_set_points has not been called");
    // inputs for the timed calls: every instance's coefficients and values in one device block
    // (filled with a finite nonzero pattern), released before returning
    int64_t nc = 0, nv = 0;
    for (int i = 0; i < b->n; ++i) { nc += b->plans[i]->Nc; nv += std::max<int64_t>(b->plans[i]->M, 1); }
    void *blk = nullptr;
    cudaError_t e = sgl::device_malloc(&blk, sizeof(double2) * (size_t)(nc + nv));
    if (e != cudaSuccess) return sgl::set_error(SGL_ERR_ALLOC, std::string("autotune inputs: ") + cudaGetErrorString(e));
    std::vector<double *> cp(b->n), vp(b->n);
    {
        double2 *c = (double2 *)blk, *v = c + nc;
        for (int i = 0; i < b->n; ++i) {
            cp[i] = (double *)c;
            vp[i] = (double *)v;
            c += b->plans[i]->Nc;
            v += std::max<int64_t>(b->plans[i]->M, 1);
        }
    }
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaMemsetAsync(blk, 0x3f, sizeof(double2) * (size_t)(nc + nv), b->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    std::vector<std::pair<int, double>> ms;
    sgl_status st = SGL_OK;
    const int orig = b->lanes;
    for (int cand : {1, 2, 4, 8, 16, 32}) {
        if (e != cudaSuccess || st != SGL_OK) break;
        if (cand > std::min(b->n, kMaxLanes)) break;
        if ((st = sgl_batch_set_lanes(b, cand)) != SGL_OK) break;
        float tot = 0.f;
        for (int it = 0; it < 5 && st == SGL_OK && e == cudaSuccess; ++it) {
            if (it == 2) e = cudaEventRecord(t0, b->stream);          // two untimed calls, then three timed
            if (e == cudaSuccess) st = sgl_batch_forward(b, cp.data(), vp.data());
            if (st == SGL_OK) st = sgl_batch_adjoint(b, vp.data(), cp.data());
        }
        if (e == cudaSuccess && st == SGL_OK) e = cudaEventRecord(t1, b->stream);
        if (e == cudaSuccess && st == SGL_OK) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess && st == SGL_OK) e = cudaEventElapsedTime(&tot, t0, t1);
        if (e == cudaSuccess && st == SGL_OK) ms.push_back({cand, tot / 3.0});
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaStreamSynchronize(b->stream);
    cudaFree(blk);
    if (st == SGL_OK && e != cudaSuccess) st = cuda_err(e, "autotune");
    if (st != SGL_OK || ms.empty()) {
        sgl_batch_set_lanes(b, std::max(1, orig));
        return st != SGL_OK ? st : sgl::set_error(SGL_ERR_CUDA, "autotune: no candidate timed");
    }
    const auto best = *std::min_element(ms.begin(), ms.end(), [](const auto &x, const auto &y) { return x.second < y.second; });
    if ((st = sgl_batch_set_lanes(b, best.first)) != SGL_OK) return st;
    if (cache_path && !cache_store(cache_path, key, best.first, ms))
        return sgl::set_error(SGL_ERR_ARG, std::string("autotune: cannot write the cache file ") + cache_path);
    if (lanes_out) *lanes_out = best.first;
    if (ms_out) *ms_out = best.second;
    return sgl::set_error(SGL_OK, "");
}

}  // extern "C"
