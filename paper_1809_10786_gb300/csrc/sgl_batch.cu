// sgl_batch.cu -- many independent transforms (each its own B, points and coefficients)
// issued together: one plan per instance, all on the batch's stream, sharing the two FFT
// work buffers (the instances run one after another in stream order).  A batch call can be
// captured into a CUDA graph once and replayed while the pointers and point counts match.
#include "sgl_internal.cuh"

#include <algorithm>
#include <new>
#include <string>
#include <vector>

struct sgl_batch {
    int n = 0;
    cudaStream_t stream = nullptr;
    std::vector<sgl_plan *> plans;
    void *bufA = nullptr, *bufB = nullptr;
    size_t bytesA = 0, bytesB = 0;
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

sgl_status fail_batch(sgl_batch *b, sgl_status st, const std::string &msg) {
    if (b) {
        for (sgl_plan *p : b->plans) sgl_plan_destroy(p);
        for (auto &e : b->exec)
            if (e) cudaGraphExecDestroy(e);
        if (b->bufA) cudaFree(b->bufA);
        if (b->bufB) cudaFree(b->bufB);
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        if (b->ev_in) cudaEventDestroy(b->ev_in);
        if (b->ev_out) cudaEventDestroy(b->ev_out);
        delete b;
    }
    return sgl::set_error(st, msg);
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

// issue every instance's call on the batch stream
sgl_status issue(sgl_batch *b, int kind, const double *const *in, double *const *out) {
    for (int i = 0; i < b->n; ++i) {
        sgl_status st = kind == 0 ? sgl_forward(b->plans[i], in[i], out[i]) : sgl_adjoint(b->plans[i], in[i], out[i]);
        if (st != SGL_OK) return st;
    }
    return SGL_OK;
}

sgl_status run(sgl_batch *b, int kind, const double *const *in, double *const *out) {
    if (!b) return sgl::set_error(SGL_ERR_ARG, "batch is NULL");
    if (!in || !out) return sgl::set_error(SGL_ERR_ARG, "pointer arrays must not be NULL");
    for (int i = 0; i < b->n; ++i)
        if (!b->plans[i]->points_set) return sgl::set_error(SGL_ERR_STATE, "sgl_batch_set_points has not been called");
    if (!b->use_graph) return issue(b, kind, in, out);
    std::vector<uintptr_t> k = make_key(b, (const void *const *)in, (const void *const *)out);
    cudaError_t e = cudaEventRecord(b->ev_in, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap_stream, b->ev_in, 0);
    if (e != cudaSuccess) return sgl::set_error(SGL_ERR_CUDA, std::string("stream ordering: ") + cudaGetErrorString(e));
    if (!b->exec[kind] || k != b->key[kind]) {
        if (b->exec[kind]) {
            cudaGraphExecDestroy(b->exec[kind]);
            b->exec[kind] = nullptr;
        }
        for (sgl_plan *p : b->plans) sgl_set_stream(p, b->cap_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed);
        sgl_status st = SGL_OK;
        if (e == cudaSuccess) {
            st = issue(b, kind, in, out);
            e = cudaStreamEndCapture(b->cap_stream, &graph);
        }
        for (sgl_plan *p : b->plans) sgl_set_stream(p, b->stream);
        if (st != SGL_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return sgl::set_error(SGL_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec[kind], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec[kind] = nullptr;
            return sgl::set_error(SGL_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
        b->key[kind] = std::move(k);
    }
    e = cudaGraphLaunch(b->exec[kind], b->cap_stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->cap_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_out, 0);
    if (e != cudaSuccess) return sgl::set_error(SGL_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    b->graph_launches += 1;
    return sgl::set_error(SGL_OK, "");
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
    for (int i = 0; i < n; ++i) {
        size_t a = 0, c = 0;
        if (sgl::plan_work_sizes(B[i], precision, q, sigma, &a, &c) != SGL_OK)
            return fail_batch(b, SGL_ERR_ARG, "instance " + std::to_string(i) + ": invalid B, q or sigma");
        b->bytesA = std::max(b->bytesA, a);
        b->bytesB = std::max(b->bytesB, c);
    }
    cudaError_t e = sgl::device_malloc(&b->bufA, b->bytesA);
    if (e == cudaSuccess) e = sgl::device_malloc(&b->bufB, b->bytesB);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail_batch(b, SGL_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    sgl::SharedWork sw{b->bufA, b->bufB, b->bytesA, b->bytesB};
    b->plans.reserve(n);
    for (int i = 0; i < n; ++i) {
        sgl_plan *p = nullptr;
        sgl_status st = sgl::plan_create_impl(&p, B[i], M_max[i], precision, window, q, sigma, flags, cuda_stream, &sw);
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
    for (auto &e : b->exec)
        if (e) cudaGraphExecDestroy(e);
    cudaStreamSynchronize(b->cap_stream);
    cudaFree(b->bufA);
    cudaFree(b->bufB);
    cudaStreamDestroy(b->cap_stream);
    cudaEventDestroy(b->ev_in);
    cudaEventDestroy(b->ev_out);
    delete b;
}

sgl_status sgl_batch_use_graph(sgl_batch *b, int enable) {
    if (!b) return sgl::set_error(SGL_ERR_ARG, "batch is NULL");
    b->use_graph = enable != 0;
    return sgl::set_error(SGL_OK, "");
}

sgl_status sgl_batch_set_points(sgl_batch *b, const double *const *xyz_dev, const int64_t *M) {
    if (!b) return sgl::set_error(SGL_ERR_ARG, "batch is NULL");
    if (!xyz_dev || !M) return sgl::set_error(SGL_ERR_ARG, "pointer arrays must not be NULL");
    for (int i = 0; i < b->n; ++i) {
        sgl_status st = sgl_set_points(b->plans[i], xyz_dev[i], M[i]);
        if (st != SGL_OK) return sgl::set_error(st, "instance " + std::to_string(i) + ": " + sgl_last_error());
    }
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
        int64_t tot = (int64_t)(b->bytesA + b->bytesB);
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
    return SGL_OK;
}

}  // extern "C"
