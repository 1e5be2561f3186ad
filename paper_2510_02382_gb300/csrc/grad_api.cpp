// Host side of the differentiable form: ctfmnmf_grad_*.
//
// The object holds one solver handle per mixture and a batch over them (so the forward pass
// is the batched path of batch_api.cpp), the checkpoints, the per-iteration state of one
// segment, and the gradient buffers of grad.cuh.
//
// forward:  load X, T0, V0 -> checkpoint 0 -> for every segment but the last: iterate
//           ckpt_every iterations, checkpoint; the last segment one iteration at a time,
//           keeping the state before each iteration and sigma (the tape) -> separated images.
// backward: images adjoint on the final state; then for segments last .. first: unless the
//           segment is on the tape, restore its checkpoint and recompute it one iteration at a
//           time the same way; then reverse its iterations. Finally the gradients of the
//           first state go to X, T0, V0.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <utility>
#include <vector>

#include "grad.cuh"
#include "handle.h"

namespace ctf {
cudaError_t batch_enqueue(ctfmnmf_batch_t b, int n_iter, cudaStream_t st);   // batch_api.cpp
}

using ctf::GradBufs;
using ctf::StatePtrs;

struct ctfmnmf_grad {
    Shape s;
    int S, K, C, nseg;
    std::vector<ctfmnmf_t> hs;
    ctfmnmf_batch_t batch;
    cudaStream_t stream;
    StatePtrs* tab;              // device [(C + 1) * S]: iteration slots 0..C-1, slot C = live state
    StatePtrs* ck;               // device [nseg * S]: checkpoints
    ctf::MixDesc* mix;           // device [S]
    GradBufs g;
    float* sig;                  // device [C][S][M]
    std::vector<void*> allocs;
    bool forwarded;
    bool taped;                  // the iteration slots hold the last segment of the forward pass
    long long launches;
    // CUDA graphs of the fixed launch sequences, captured on first use on a private stream and
    // replayed on the object's stream: a recorded segment by length (the checkpoint length and
    // the last segment's), the reverse pass of each segment; with their kernel counts
    cudaStream_t cap;
    cudaGraphExec_t rec_graph[2];
    int rec_len[2];
    long long rec_kernels[2];
    std::vector<cudaGraphExec_t> rev_graph;
    std::vector<long long> rev_kernels;
};

namespace {

int gfail(int code, const char* fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctf::set_thread_error(buf);
    return code;
}

template <typename T>
bool dalloc(ctfmnmf_grad* g, T** p, size_t count)
{
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    g->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return true;
}

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Byte offsets of (Y, W, T, V) inside one state block and the block size.
struct BlockLayout {
    size_t y, w, t, v, size;
};
BlockLayout block_layout(const Shape& s)
{
    BlockLayout L;
    L.y = 0;
    L.w = L.y + al256(sizeof(float2) * (size_t)s.F * s.M * s.Jp);
    L.t = L.w + al256(sizeof(float2) * (size_t)s.F * s.M * s.M);
    L.v = L.t + al256(sizeof(float) * (size_t)s.N * s.FBp);
    L.size = L.v + al256(sizeof(float) * (size_t)s.N * s.B * s.Jp);
    return L;
}

StatePtrs block_ptrs(char* base, const BlockLayout& L)
{
    StatePtrs p;
    p.Y = reinterpret_cast<float2*>(base + L.y);
    p.W = reinterpret_cast<float2*>(base + L.w);
    p.T = reinterpret_cast<float*>(base + L.t);
    p.V = reinterpret_cast<float*>(base + L.v);
    return p;
}

int seg_len(const ctfmnmf_grad* g, int c) { return c + 1 < g->nseg ? g->C : g->K - c * g->C; }

// Capture enqueue(stream) -> kernel count (< 0: failure) into *slot on the capture stream once,
// then launch the graph on st. Returns the kernel count, or -1.
template <class Fn>
long long graph_run(ctfmnmf_grad* g, cudaGraphExec_t* slot, long long* kernels, Fn enqueue, cudaStream_t st)
{
    if (!*slot) {
        cudaGraph_t gr = nullptr;
        if (cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -1;
        const long long n = enqueue(g->cap);
        const cudaError_t ec = cudaStreamEndCapture(g->cap, &gr);
        if (n < 0 || ec != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
            return -1;
        }
        const cudaError_t ei = cudaGraphInstantiate(slot, gr, 0);
        cudaGraphDestroy(gr);
        if (ei != cudaSuccess) {
            *slot = nullptr;
            return -1;
        }
        *kernels = n;
    }
    return cudaGraphLaunch(*slot, st) == cudaSuccess ? *kernels : -1;
}

// Run `len` iterations from the live state one at a time, keeping the state before each one in
// iteration slot t and the applied normalisation in sigma slot t: slot 0 by a copy, slot t + 1
// by the finalize of iteration t. Returns the number of launches, or -1 on a launch failure.
long long record_segment_direct(ctfmnmf_grad* g, int len, cudaStream_t st)
{
    const Shape& s = g->s;
    const int S = g->S;
    const StatePtrs* live = g->tab + (size_t)g->C * S;
    if (ctf::grad_launch_copy(s, S, live, g->tab, st) != cudaSuccess) return -1;
    long long n = 1;
    for (int t = 0; t < len; ++t) {
        const StatePtrs* snap = t + 1 < len ? g->tab + (size_t)(t + 1) * S : nullptr;
        if (ctf::batch_enqueue(g->batch, 1, st) != cudaSuccess ||
            ctf::grad_launch_finalize(s, S, g->mix, g->sig + (size_t)t * S * s.M, st, snap) != cudaSuccess)
            return -1;
        n += snap ? 1 : 2;                              // finalize (+ scale reset after the last)
    }
    int info[5] = {0, 0, 0, 0, 0};
    ctfmnmf_batch_info(g->batch, info);
    return n + (long long)len * (info[1] + info[2]);
}

// record_segment_direct through a graph per segment length
long long record_segment(ctfmnmf_grad* g, int len, cudaStream_t st)
{
    int k = 0;
    while (k < 2 && g->rec_graph[k] && g->rec_len[k] != len) ++k;
    if (k == 2) return record_segment_direct(g, len, st);   // not expected: two lengths at most
    g->rec_len[k] = len;
    return graph_run(g, &g->rec_graph[k], &g->rec_kernels[k],
                     [&](cudaStream_t cs) { return record_segment_direct(g, len, cs); }, st);
}

void release(ctfmnmf_grad* g)
{
    for (int k = 0; k < 2; ++k)
        if (g->rec_graph[k]) cudaGraphExecDestroy(g->rec_graph[k]);
    for (cudaGraphExec_t x : g->rev_graph)
        if (x) cudaGraphExecDestroy(x);
    if (g->cap) cudaStreamDestroy(g->cap);
    if (g->batch) ctfmnmf_batch_destroy(g->batch);
    for (ctfmnmf_t h : g->hs) ctfmnmf_destroy(h);
    for (void* p : g->allocs) cudaFree(p);
    delete g;
}

long long batch_launches(ctfmnmf_batch_t b)
{
    int info[5] = {0, 0, 0, 0, 0};
    ctfmnmf_batch_info(b, info);
    return info[4];
}

}  // namespace

extern "C" {

int ctfmnmf_grad_create(const ctfmnmf_dims* dims, const int* Ln, int batch, int n_iter, int ckpt_every,
                        ctfmnmf_grad_t* out)
{
    ctf::set_thread_error("");
    if (!out) return gfail(CTFMNMF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!dims) return gfail(CTFMNMF_EINVAL, "dims is NULL");
    if (batch < 1 || n_iter < 1 || ckpt_every < 1)
        return gfail(CTFMNMF_EINVAL, "need batch >= 1, n_iter >= 1 and ckpt_every >= 1");
    if (dims->M < 2 || dims->M > ctf::kGradMaxM)
        return gfail(dims->M > 0 ? CTFMNMF_EUNSUPPORTED : CTFMNMF_EINVAL,
                     "the differentiable form supports 2 <= M <= %d (M=%d)", ctf::kGradMaxM, dims->M);
    if (dims->J > ctf::kGradMaxJ)
        return gfail(CTFMNMF_EUNSUPPORTED, "the differentiable form supports J <= %d (J=%d)", ctf::kGradMaxJ,
                     dims->J);
    ctfmnmf_grad* g = new (std::nothrow) ctfmnmf_grad;
    if (!g) return gfail(CTFMNMF_ENOMEM, "host allocation failed");
    g->S = batch;
    g->K = n_iter;
    g->C = ckpt_every < n_iter ? ckpt_every : n_iter;
    g->nseg = (n_iter + g->C - 1) / g->C;
    g->batch = nullptr;
    g->stream = nullptr;
    g->tab = nullptr;
    g->ck = nullptr;
    g->mix = nullptr;
    g->sig = nullptr;
    g->forwarded = false;
    g->taped = false;
    g->launches = 0;
    g->cap = nullptr;
    for (int k = 0; k < 2; ++k) {
        g->rec_graph[k] = nullptr;
        g->rec_len[k] = 0;
        g->rec_kernels[k] = 0;
    }
    g->rev_graph.assign(g->nseg, nullptr);
    g->rev_kernels.assign(g->nseg, 0);
    memset(&g->g, 0, sizeof(g->g));
    ctfmnmf_options opt;
    ctfmnmf_default_options(&opt);
    opt.path = CTFMNMF_PATH_TWO_KERNEL;          // the batched kernels run the iterations
    for (int k = 0; k < batch; ++k) {
        ctfmnmf_t h = nullptr;
        const int rc = ctfmnmf_create_ex(dims, Ln, &opt, &h);
        if (rc != CTFMNMF_OK) {
            char msg[256];
            snprintf(msg, sizeof(msg), "%s", ctfmnmf_last_error(nullptr));
            release(g);
            return gfail(rc, "%s", msg);
        }
        g->hs.push_back(h);
    }
    const Shape& s = g->hs[0]->s;
    g->s = s;
    const int S = g->S, M = s.M, N = s.N, F = s.F, B = s.B, Jp = s.Jp;
    const BlockLayout L = block_layout(s);
    char* stash = nullptr;
    char* ckm = nullptr;
    GradBufs& gb = g->g;
    const size_t nY = (size_t)S * F * M * Jp, nT = (size_t)S * N * s.FBp, nV = (size_t)S * N * B * Jp,
                 nL = (size_t)S * N * F * Jp;
    bool ok = dalloc(g, &stash, L.size * g->C * S) && dalloc(g, &ckm, L.size * g->nseg * S) &&
              dalloc(g, &g->tab, (size_t)(g->C + 1) * S) && dalloc(g, &g->ck, (size_t)g->nseg * S) &&
              dalloc(g, &g->mix, (size_t)S) && dalloc(g, &g->sig, (size_t)g->C * S * M) &&
              dalloc(g, &gb.gY, nY) && dalloc(g, &gb.gW, (size_t)S * F * M * M) && dalloc(g, &gb.gT, nT) &&
              dalloc(g, &gb.gV[0], nV) && dalloc(g, &gb.gV[1], nV) && dalloc(g, &gb.gnum, nV) &&
              dalloc(g, &gb.gden, nV) && dalloc(g, &gb.glp, nL) && dalloc(g, &gb.glt, nL) &&
              dalloc(g, &gb.aq, nL) && dalloc(g, &gb.gsa, nL) && dalloc(g, &gb.ilp, nL) && dalloc(g, &gb.actp, ctf::grad_act_partials(s, S)) &&
              dalloc(g, &gb.gnT, nT) && dalloc(g, &gb.gdT, nT) &&
              dalloc(g, &gb.e, (size_t)S * M) && dalloc(g, &gb.e_prev, (size_t)S * M);
    if (!ok) {
        release(g);
        return gfail(CTFMNMF_ENOMEM, "device allocation of the differentiable form failed");
    }
    std::vector<StatePtrs> htab((size_t)(g->C + 1) * S), hck((size_t)g->nseg * S);
    std::vector<ctf::MixDesc> hmix(S);
    for (int c = 0; c < g->C; ++c)
        for (int k = 0; k < S; ++k) htab[(size_t)c * S + k] = block_ptrs(stash + L.size * ((size_t)c * S + k), L);
    for (int k = 0; k < S; ++k) {
        const State& d = g->hs[k]->d;
        htab[(size_t)g->C * S + k] = StatePtrs{d.Y, d.W, d.T, d.V};
        hmix[k].s = g->hs[k]->s;
        hmix[k].d = d;
    }
    for (int c = 0; c < g->nseg; ++c)
        for (int k = 0; k < S; ++k) hck[(size_t)c * S + k] = block_ptrs(ckm + L.size * ((size_t)c * S + k), L);
    if (cudaMemcpy(g->tab, htab.data(), sizeof(StatePtrs) * htab.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->ck, hck.data(), sizeof(StatePtrs) * hck.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->mix, hmix.data(), sizeof(ctf::MixDesc) * S, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        release(g);
        return gfail(CTFMNMF_ECUDA, "copying the state tables to the device failed");
    }
    if (cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        g->cap = nullptr;
        release(g);
        return gfail(CTFMNMF_ECUDA, "creating the capture stream failed");
    }
    const cudaError_t e = ctf::grad_configure(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(g);
        return gfail(CTFMNMF_EUNSUPPORTED, "the per-bin adjoint kernel cannot be configured for this shape: %s",
                     cudaGetErrorString(e));
    }
    *out = g;
    return CTFMNMF_OK;
}

int ctfmnmf_grad_set_stream(ctfmnmf_grad_t g, void* stream)
{
    ctf::set_thread_error("");
    if (!g) return gfail(CTFMNMF_EINVAL, "object is NULL");
    g->stream = (cudaStream_t)stream;
    for (ctfmnmf_t h : g->hs) ctfmnmf_set_stream(h, stream);
    return CTFMNMF_OK;
}

int ctfmnmf_grad_forward(ctfmnmf_grad_t g, const void* X, const float* T0, const float* V0, void* C)
{
    ctf::TraceRange trace("ctfmnmf_grad_forward");
    ctf::set_thread_error("");
    if (!g) return gfail(CTFMNMF_EINVAL, "object is NULL");
    if (!X || !T0 || !V0 || !C) return gfail(CTFMNMF_EINVAL, "null pointer argument");
    const Shape& s = g->s;
    const int S = g->S;
    cudaStream_t st = g->stream;
    g->forwarded = false;
    for (int k = 0; k < S; ++k) {
        ctfmnmf* h = g->hs[k];
        const float2* Xk = static_cast<const float2*>(X) + (size_t)k * s.M * s.F * s.J;
        if (ctf::launch_load(h->s, h->d, Xk, st) != cudaSuccess ||
            ctf::launch_init_nmf(h->s, h->d, T0 + (size_t)k * s.N * s.F * s.B, V0 + (size_t)k * s.N * s.B * s.J, 0,
                                 st) != cudaSuccess ||
            ctf::launch_psd(h->s, h->d, st) != cudaSuccess)
            return gfail(CTFMNMF_ECUDA, "loading mixture %d failed", k);
        h->loaded = true;
    }
    g->launches += 3LL * S;
    if (!g->batch) {
        const int rc = ctfmnmf_batch_create(S, g->hs.data(), &g->batch);
        if (rc != CTFMNMF_OK) return rc;
    }
    if (ctf::grad_launch_copy(s, S, g->tab + (size_t)g->C * S, g->ck, st) != cudaSuccess)
        return gfail(CTFMNMF_ECUDA, "checkpoint copy failed");
    ++g->launches;
    g->taped = false;
    const long long b0 = batch_launches(g->batch);
    for (int c = 0; c + 1 < g->nseg; ++c) {
        const int rc = ctfmnmf_batch_iterate(g->batch, seg_len(g, c));
        if (rc != CTFMNMF_OK) return rc;
        if (ctf::grad_launch_copy(s, S, g->tab + (size_t)g->C * S, g->ck + (size_t)(c + 1) * S, st) != cudaSuccess)
            return gfail(CTFMNMF_ECUDA, "checkpoint copy failed");
        ++g->launches;
    }
    g->launches += batch_launches(g->batch) - b0;
    const long long nrec = record_segment(g, seg_len(g, g->nseg - 1), st);
    if (nrec < 0) return gfail(CTFMNMF_ECUDA, "the last segment's iterations failed");
    g->launches += nrec;
    g->taped = true;
    for (int k = 0; k < S; ++k) {
        ctfmnmf* h = g->hs[k];
        float2* Ck = static_cast<float2*>(C) + (size_t)k * s.N * s.M * s.F * s.J;
        if (ctf::launch_separate(h->s, h->d, Ck, st) != cudaSuccess)
            return gfail(CTFMNMF_ECUDA, "images of mixture %d failed", k);
    }
    g->launches += S;
    g->forwarded = true;
    return CTFMNMF_OK;
}

int ctfmnmf_grad_backward(ctfmnmf_grad_t g, const void* gC, void* gX, float* gT0, float* gV0)
{
    ctf::TraceRange trace("ctfmnmf_grad_backward");
    ctf::set_thread_error("");
    if (!g) return gfail(CTFMNMF_EINVAL, "object is NULL");
    if (!gC || !gX || !gT0 || !gV0) return gfail(CTFMNMF_EINVAL, "null pointer argument");
    if (!g->forwarded) return gfail(CTFMNMF_ESTATE, "no forward pass to differentiate");
    const Shape& s = g->s;
    const int S = g->S, M = s.M;
    cudaStream_t st = g->stream;
    const StatePtrs* live = g->tab + (size_t)g->C * S;
    GradBufs gb = g->g;
    gb.sig = g->sig;
    if (ctf::grad_launch_head(s, S, live, static_cast<const float2*>(gC), gb, st) != cudaSuccess ||
        cudaMemsetAsync(gb.gV[0], 0, sizeof(float) * (size_t)S * s.N * s.B * s.Jp, st) != cudaSuccess)
        return gfail(CTFMNMF_ECUDA, "images adjoint failed");
    long long n = 1;
    int gcur = 0, ecur = 0;
    bool first = true;
    // the forward state is consumed from here on: a second backward needs a new forward
    g->forwarded = false;
    const bool taped = g->taped;
    g->taped = false;
    for (int c = g->nseg - 1; c >= 0; --c) {
        const int len = seg_len(g, c);
        if (!(taped && c == g->nseg - 1)) {
            if (ctf::grad_launch_copy(s, S, g->ck + (size_t)c * S, g->tab + (size_t)g->C * S, st) != cudaSuccess)
                return gfail(CTFMNMF_ECUDA, "restoring checkpoint %d failed", c);
            for (ctfmnmf_t h : g->hs)
                if (ctf::launch_psd(h->s, h->d, st) != cudaSuccess) return gfail(CTFMNMF_ECUDA, "psd launch failed");
            n += 1 + S;
            const long long nrec = record_segment(g, len, st);
            if (nrec < 0) return gfail(CTFMNMF_ECUDA, "recomputing segment %d failed", c);
            n += nrec;
        }
        // the reverse pass of the segment: a fixed sequence for a given segment (the buffer
        // parities and `first` follow from the iterations reversed before it)
        const int gcur0 = gcur, ecur0 = ecur;
        const bool first0 = first;
        auto reverse = [&](cudaStream_t rs) -> long long {
            int gc = gcur0, ec = ecur0;
            bool fst = first0;
            long long nk = 0;
            for (int t = len - 1; t >= 0; --t) {
                GradBufs gi = g->g;
                gi.sig = g->sig + (size_t)t * S * M;
                if (ec) std::swap(gi.e, gi.e_prev);    // the sums written by the previous iteration
                const StatePtrs* cur = g->tab + (size_t)t * S;
                const StatePtrs* nxt = t + 1 == len ? live : g->tab + (size_t)(t + 1) * S;
                int kernels = 0;
                if (ctf::grad_enqueue_iteration(s, S, cur, nxt, gi, gc, fst, rs, &kernels) != cudaSuccess) return -1;
                gc = 1 - gc;
                ec = 1 - ec;
                fst = false;
                nk += kernels;
            }
            return nk;
        };
        const long long nrev = graph_run(g, &g->rev_graph[c], &g->rev_kernels[c], reverse, st);
        if (nrev < 0) return gfail(CTFMNMF_ECUDA, "backward of segment %d failed", c);
        n += nrev;
        if (len & 1) {
            gcur = 1 - gcur;
            ecur = 1 - ecur;
        }
        first = false;
    }
    if (ctf::grad_launch_inputs(s, S, g->ck, g->g, gcur, static_cast<float2*>(gX), gT0, gV0, st) != cudaSuccess)
        return gfail(CTFMNMF_ECUDA, "input gradients failed");
    g->launches += n + 2;
    return CTFMNMF_OK;
}

int ctfmnmf_grad_mse(ctfmnmf_grad_t g, const void* C, const void* Cref, double* loss, const double* dloss, void* gC)
{
    ctf::set_thread_error("");
    if (!g) return gfail(CTFMNMF_EINVAL, "object is NULL");
    if (!C || !Cref) return gfail(CTFMNMF_EINVAL, "null pointer argument");
    if (!loss && !gC) return CTFMNMF_OK;
    const Shape& s = g->s;
    const size_t count = (size_t)g->S * s.N * s.M * s.F * s.J;
    if (ctf::grad_launch_mse(count, static_cast<const float2*>(C), static_cast<const float2*>(Cref), loss, dloss,
                             static_cast<float2*>(gC), g->stream) != cudaSuccess)
        return gfail(CTFMNMF_ECUDA, "loss kernel failed");
    ++g->launches;
    return CTFMNMF_OK;
}

int ctfmnmf_grad_launch_count(ctfmnmf_grad_t g, long long* count)
{
    ctf::set_thread_error("");
    if (!g || !count) return gfail(CTFMNMF_EINVAL, "need an object and an output");
    *count = g->launches;
    return CTFMNMF_OK;
}

int ctfmnmf_grad_destroy(ctfmnmf_grad_t g)
{
    if (!g) return CTFMNMF_OK;
    cudaStreamSynchronize(g->stream);
    release(g);
    return CTFMNMF_OK;
}

}  // extern "C"
