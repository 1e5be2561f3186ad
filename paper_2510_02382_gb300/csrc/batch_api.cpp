// Host side of the batched path: ctfmnmf_batch_create / _iterate / _time / _destroy.
//
// A batch groups solver handles of one device. Their mixtures are sorted into launch
// classes: bin classes by (M, frames per thread, threads per block) and frame classes by
// the width of the bases arrays. One iteration = one bin-phase launch per bin class, then
// one frame-phase launch per frame class; n iterations are captured once into a CUDA graph
// and replayed. The autotuner picks the class plan: for each candidate (frames-per-thread
// preference x whether classes of one (M, frames per thread) share the largest block) it
// times two iterations on the handles' buffers, with the evolving state saved before and
// restored after, so creating a batch leaves every handle unchanged.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "handle.h"

using ctf::BatchClass;
using ctf::MixDesc;

namespace {

struct FrameClass {
    int BB, exact, blocks;       // exact: every mixture of the class has B == BB
    int2* work;
};

struct Plan {
    std::vector<BatchClass> bins;
    std::vector<FrameClass> frames;
};

void free_plan(Plan& p)
{
    for (auto& c : p.bins)
        if (c.work) cudaFree(c.work);
    for (auto& c : p.frames)
        if (c.work) cudaFree(c.work);
    p.bins.clear();
    p.frames.clear();
}

// Frames per thread and threads per block of a mixture under a preference: 0 = the
// single-mixture choice (fewest frames per thread within 256 threads), 1 = 8 frames per
// thread wherever M <= 4 allows it.
bool bin_shape(int M, int J, int pref, int* fpt, int* nt)
{
    if (pref == 1 && M <= 4) {
        const int t = ((J + 7) / 8 + 31) / 32 * 32;
        if (t <= 512) {
            *fpt = 8;
            *nt = t < 64 ? 64 : t;
            return true;
        }
    }
    return ctf::bin_phase_config(M, J, fpt, nt);
}

// pref 2: the contiguous-frame bin phase (ctf::kBinContig) for every mixture it supports
// (M <= 4, default taps), preference 1 for the others.
int make_plan(const std::vector<ctfmnmf*>& hs, int pref, bool merge, Plan* out)
{
    // key -> list of (mixture, F) ; key = (M, fpt, nt with 0 when merged, bases class, or
    // 1000 + 16 N + bases groups for the contiguous-frame classes, compiled per N and groups)
    std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
    std::vector<int> mix_nt(hs.size());
    for (size_t b = 0; b < hs.size(); ++b) {
        const Shape& s = hs[b]->s;
        int fpt = 0, nt = 0;
        if (pref == 2 && ctf::contig_supported(s)) {
            fpt = ctf::kBinContig;
            nt = ctf::contig_threads(s);
        } else if (!bin_shape(s.M, s.J, pref == 2 ? 1 : pref, &fpt, &nt)) {
            return CTFMNMF_EUNSUPPORTED;
        }
        mix_nt[b] = nt;
        const int sub = fpt == ctf::kBinContig ? 1000 + 16 * s.N + ctf::contig_groups(s.B) : ctf::bases_class(s.B);
        groups[std::make_tuple(s.M, fpt, merge ? 0 : nt, sub)].push_back((int)b);
    }
    for (auto& kv : groups) {
        BatchClass c;
        memset(&c, 0, sizeof(c));
        c.M = std::get<0>(kv.first);
        c.fpt = std::get<1>(kv.first);
        const bool contig = c.fpt == ctf::kBinContig;
        c.kb = contig ? (std::get<3>(kv.first) - 1000) % 16 : std::get<3>(kv.first);
        c.N = contig ? (std::get<3>(kv.first) - 1000) / 16 : 0;
        int nt = 0;
        size_t smem = 0;
        std::vector<int2> work;
        for (int b : kv.second) nt = std::max(nt, mix_nt[b]);
        for (int b : kv.second) {
            const Shape& s = hs[b]->s;
            smem = std::max(smem, contig ? ctf::contig_smem_bytes(s, nt)
                                         : sizeof(float) * (size_t)ctf::bin_smem_floats(s, nt));
            for (int i = 0; i < s.F; ++i) work.push_back(make_int2(b, i));
        }
        c.nt = nt;
        c.smem = smem;
        c.blocks = (int)work.size();
        if (cudaMalloc((void**)&c.work, sizeof(int2) * work.size()) != cudaSuccess ||
            cudaMemcpy(c.work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            out->bins.push_back(c);
            return CTFMNMF_ENOMEM;
        }
        out->bins.push_back(c);
    }
    std::map<int, std::vector<int2>> fwork;
    for (size_t b = 0; b < hs.size(); ++b) {
        const Shape& s = hs[b]->s;
        const int BB = ctf::batch_frame_class(s.B);
        if (ctf::batch_frame_chunk(s.B, BB) < 4) return CTFMNMF_EUNSUPPORTED;
        const int items = (s.Jp / 8) * s.N;
        const int key = 2 * BB + (s.B == BB ? 1 : 0);     // mixtures whose B is the class width apart
        fwork[key].push_back(make_int2((int)b, -1));       // the mixture's normalisation scale
        for (int it = 0; it < items; ++it) fwork[key].push_back(make_int2((int)b, it));
    }
    for (auto& kv : fwork) {
        FrameClass f;
        f.BB = kv.first / 2;
        f.exact = kv.first & 1;
        f.blocks = (int)kv.second.size();
        f.work = nullptr;
        if (cudaMalloc((void**)&f.work, sizeof(int2) * kv.second.size()) != cudaSuccess ||
            cudaMemcpy(f.work, kv.second.data(), sizeof(int2) * kv.second.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            cudaGetLastError();
            out->frames.push_back(f);
            return CTFMNMF_ENOMEM;
        }
        out->frames.push_back(f);
    }
    return CTFMNMF_OK;
}

}  // namespace

constexpr int kBranches = 4;     // concurrent bin-class branches per iteration

struct ctfmnmf_batch {
    std::vector<ctfmnmf*> hs;
    MixDesc* dmix;              // device [count]
    Plan plan;
    int policy;                 // chosen candidate: 2 * pref + merge (pref 2: contiguous frames)
    int v_tap0, normalize;
    cudaStream_t capture;
    cudaGraphExec_t graph;
    int graph_iters;
    long long launches;
    // the bin classes of one iteration touch disjoint mixtures: they run as parallel
    // branches (side streams forked from and joined to the launching stream by events)
    cudaStream_t side[kBranches];
    cudaEvent_t fork, join[kBranches];
};

namespace {

void release_branches(ctfmnmf_batch* b)
{
    for (int k = 0; k < kBranches; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
}

int fail_b(int code, const char* fmt, const char* what = "")
{
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, what);
    ctf::set_thread_error(buf);
    return code;
}

cudaError_t enqueue_batch(ctfmnmf_batch* b, const Plan& p, int n_iter, cudaStream_t st)
{
    const int nb = (int)p.bins.size();
    const int K = nb < kBranches ? nb : kBranches;
    for (int t = 0; t < n_iter; ++t) {
        if (K > 1) {
            // fork: class c on branch c % K; join before the frame phase, which reads every
            // mixture's bin-phase output
            cudaError_t e = cudaEventRecord(b->fork, st);
            for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
            for (int c = 0; c < nb && e == cudaSuccess; ++c)
                e = ctf::launch_batch_bin(p.bins[c], b->dmix, b->v_tap0, b->side[c % K], false);
            for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaEventRecord(b->join[k], b->side[k]);
            for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(st, b->join[k], 0);
            if (e != cudaSuccess) return e;
        } else {
            for (const auto& c : p.bins) {
                cudaError_t e = ctf::launch_batch_bin(c, b->dmix, b->v_tap0, st, false);
                if (e != cudaSuccess) return e;
            }
        }
        for (const auto& f : p.frames) {
            cudaError_t e = ctf::launch_batch_frame(f.BB, f.exact, b->dmix, f.work, f.blocks, b->v_tap0, b->normalize, st);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t configure_plan(const Plan& p, const MixDesc* dmix)
{
    for (const auto& c : p.bins) {
        cudaError_t e = ctf::launch_batch_bin(c, dmix, 0, nullptr, true);
        if (e != cudaSuccess) return e;
    }
    return ctf::configure_batch_frame();
}

// buffers an iteration changes (P and the row powers are rewritten before use)
struct Saved {
    std::vector<std::pair<void*, size_t>> bufs;
    std::vector<void*> copies;
};

bool save_state(const std::vector<ctfmnmf*>& hs, Saved* sv, cudaStream_t st)
{
    for (ctfmnmf* h : hs) {
        const Shape& s = h->s;
        const State& d = h->d;
        const size_t MF = (size_t)s.M * s.F;
        sv->bufs.push_back({d.Y, sizeof(float2) * MF * s.Jp});
        sv->bufs.push_back({d.W, sizeof(float2) * MF * s.M});
        sv->bufs.push_back({d.T, sizeof(float) * (size_t)s.N * s.FBp});
        sv->bufs.push_back({d.V, sizeof(float) * (size_t)s.N * s.B * s.Jp});
        sv->bufs.push_back({d.invlam, sizeof(float) * (size_t)s.F * s.N * s.Jp});
        sv->bufs.push_back({d.logdet, sizeof(double) * s.F});
        sv->bufs.push_back({d.ldm, sizeof(double) * s.F});
        sv->bufs.push_back({d.lde, sizeof(int) * s.F});
        sv->bufs.push_back({d.scale, sizeof(float) * CTFMNMF_MAX_M});
    }
    for (auto& bf : sv->bufs) {
        void* c = nullptr;
        if (cudaMalloc(&c, bf.second) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        sv->copies.push_back(c);
        if (cudaMemcpyAsync(c, bf.first, bf.second, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return false;
    }
    return true;
}

void restore_state(Saved* sv, cudaStream_t st)
{
    for (size_t k = 0; k < sv->copies.size(); ++k)
        cudaMemcpyAsync(sv->bufs[k].first, sv->copies[k], sv->bufs[k].second, cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
    for (void* c : sv->copies) cudaFree(c);
    sv->copies.clear();
}

}  // namespace

extern "C" {

int ctfmnmf_batch_create(int count, const ctfmnmf_t* handles, ctfmnmf_batch_t* out)
{
    ctf::set_thread_error("");
    if (!out) return fail_b(CTFMNMF_EINVAL, "out is NULL");
    *out = nullptr;
    if (count <= 0 || !handles) return fail_b(CTFMNMF_EINVAL, "need count > 0 handles");
    int dev = 0;
    cudaGetDevice(&dev);
    for (int k = 0; k < count; ++k) {
        const ctfmnmf* h = handles[k];
        if (!h) return fail_b(CTFMNMF_EINVAL, "handle is NULL");
        if (h->device != dev) return fail_b(CTFMNMF_EINVAL, "all handles must live on the current device");
        if (h->opt.v_update != handles[0]->opt.v_update || h->opt.normalize != handles[0]->opt.normalize)
            return fail_b(CTFMNMF_EINVAL, "all handles need the same v_update and normalize options");
        for (int q = 0; q < k; ++q)
            if (handles[q] == h) return fail_b(CTFMNMF_EINVAL, "a handle appears twice");
        if (h->opt.w_update != CTFMNMF_W_ISS)
            return fail_b(CTFMNMF_EUNSUPPORTED, "the batched form runs the ISS update only");
    }
    ctfmnmf_batch* b = new (std::nothrow) ctfmnmf_batch;
    if (!b) return fail_b(CTFMNMF_ENOMEM, "host allocation failed");
    b->hs.assign(handles, handles + count);
    b->dmix = nullptr;
    b->capture = nullptr;
    b->fork = nullptr;
    for (int k = 0; k < kBranches; ++k) {
        b->side[k] = nullptr;
        b->join[k] = nullptr;
    }
    b->graph = nullptr;
    b->graph_iters = 0;
    b->launches = 0;
    b->policy = 0;
    b->v_tap0 = handles[0]->opt.v_update == CTFMNMF_V_TAP0;
    b->normalize = handles[0]->opt.normalize;
    std::vector<MixDesc> mix(count);
    for (int k = 0; k < count; ++k) {
        mix[k].s = handles[k]->s;
        mix[k].d = handles[k]->d;
    }
    int rc = CTFMNMF_OK;
    if (cudaMalloc((void**)&b->dmix, sizeof(MixDesc) * count) != cudaSuccess ||
        cudaMemcpy(b->dmix, mix.data(), sizeof(MixDesc) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        rc = fail_b(CTFMNMF_ENOMEM, "device set-up of the batch failed");
    }
    for (int k = 0; k < kBranches && rc == CTFMNMF_OK; ++k)
        if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            rc = fail_b(CTFMNMF_ENOMEM, "device set-up of the batch failed");
        }
    // ---- autotune: candidates (preference, merge), two timed iterations each
    cudaStream_t st = b->hs[0]->stream;
    Saved sv;
    if (rc == CTFMNMF_OK && !save_state(b->hs, &sv, st)) rc = fail_b(CTFMNMF_ENOMEM, "no memory to save state for tuning");
    float best = 1e30f;
    // diagnostic: CTFMNMF_BATCH_PLAN=k in the environment keeps only candidate k (0..5)
    int only = -1;
    if (const char* env = getenv("CTFMNMF_BATCH_PLAN")) {
        if (env[0] >= '0' && env[0] <= '5' && env[1] == 0) only = env[0] - '0';
    }
    for (int cand = 0; cand < 6 && rc == CTFMNMF_OK; ++cand) {
        if (only >= 0 && cand != only) continue;
        Plan p;
        const int prc = make_plan(b->hs, cand / 2, (cand & 1) != 0, &p);
        if (prc != CTFMNMF_OK || configure_plan(p, b->dmix) != cudaSuccess) {
            cudaGetLastError();
            free_plan(p);
            continue;
        }
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        bool ok = enqueue_batch(b, p, 1, st) == cudaSuccess;
        ok = ok && cudaEventRecord(e0, st) == cudaSuccess;
        ok = ok && enqueue_batch(b, p, 2, st) == cudaSuccess;
        ok = ok && cudaEventRecord(e1, st) == cudaSuccess;
        ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.f;
        if (ok) cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaGetLastError();
        if (ok && ms < best) {
            best = ms;
            free_plan(b->plan);
            b->plan = p;
            b->policy = cand;
        } else {
            free_plan(p);
        }
    }
    if (!sv.copies.empty()) restore_state(&sv, st);
    if (rc == CTFMNMF_OK && b->plan.bins.empty())
        rc = fail_b(CTFMNMF_EUNSUPPORTED, "no launch plan fits these mixtures");
    if (rc == CTFMNMF_OK && configure_plan(b->plan, b->dmix) != cudaSuccess)
        rc = fail_b(CTFMNMF_ECUDA, "configuring the chosen plan failed");
    if (rc != CTFMNMF_OK) {
        free_plan(b->plan);
        if (b->dmix) cudaFree(b->dmix);
        if (b->capture) cudaStreamDestroy(b->capture);
        release_branches(b);
        delete b;
        return rc;
    }
    *out = b;
    return CTFMNMF_OK;
}

int ctfmnmf_batch_iterate(ctfmnmf_batch_t b, int n_iter)
{
    ctf::TraceRange trace("ctfmnmf_batch_iterate");
    ctf::set_thread_error("");
    if (!b) return fail_b(CTFMNMF_EINVAL, "batch is NULL");
    if (n_iter < 0) return fail_b(CTFMNMF_EINVAL, "n_iter is negative");
    for (ctfmnmf* h : b->hs)
        if (!h->loaded) return fail_b(CTFMNMF_ESTATE, "a mixture of the batch has no STFT loaded");
    if (n_iter == 0) return CTFMNMF_OK;
    cudaStream_t st = b->hs[0]->stream;
    if (!b->graph || b->graph_iters != n_iter) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fail_b(CTFMNMF_ECUDA, "graph capture failed to start");
        const cudaError_t e = enqueue_batch(b, b->plan, n_iter, b->capture);
        const cudaError_t ec = cudaStreamEndCapture(b->capture, &g);
        if (e != cudaSuccess || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return fail_b(CTFMNMF_ECUDA, "capturing the batched iterations failed: %s",
                          cudaGetErrorString(e != cudaSuccess ? e : ec));
        }
        const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            b->graph = nullptr;
            return fail_b(CTFMNMF_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
        }
        b->graph_iters = n_iter;
    }
    if (cudaGraphLaunch(b->graph, st) != cudaSuccess) return fail_b(CTFMNMF_ECUDA, "graph launch failed");
    for (ctfmnmf* h : b->hs)
        if (ctf::launch_finalize(h->s, h->d, st) != cudaSuccess) return fail_b(CTFMNMF_ECUDA, "finalize launch failed");
    b->launches += (long long)n_iter * (long long)(b->plan.bins.size() + b->plan.frames.size()) +
                   (long long)ctf::kFinalizeKernels * (long long)b->hs.size();
    return CTFMNMF_OK;
}

int ctfmnmf_batch_time(ctfmnmf_batch_t b, int n_iter, double* ms)
{
    ctf::set_thread_error("");
    if (!b || !ms || n_iter < 1) return fail_b(CTFMNMF_EINVAL, "need a batch, n_iter >= 1 and an output");
    cudaStream_t st = b->hs[0]->stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail_b(CTFMNMF_ECUDA, "event creation failed");
    int rc = cudaEventRecord(e0, st) == cudaSuccess ? CTFMNMF_OK : CTFMNMF_ECUDA;
    if (rc == CTFMNMF_OK) rc = ctfmnmf_batch_iterate(b, n_iter);
    if (rc == CTFMNMF_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        rc = CTFMNMF_ECUDA;
    float t = 0.f;
    if (rc == CTFMNMF_OK) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CTFMNMF_OK) return rc == CTFMNMF_ECUDA ? fail_b(rc, "batch timing failed") : rc;
    *ms = t;
    return CTFMNMF_OK;
}

int ctfmnmf_batch_info(ctfmnmf_batch_t b, int* info)
{
    ctf::set_thread_error("");
    if (!b || !info) return fail_b(CTFMNMF_EINVAL, "need a batch and an output");
    info[0] = (int)b->hs.size();
    info[1] = (int)b->plan.bins.size();
    info[2] = (int)b->plan.frames.size();
    info[3] = b->policy;
    info[4] = (int)(b->launches & 0x7fffffff);
    return CTFMNMF_OK;
}

int ctfmnmf_debug_set_work(ctfmnmf_batch_t b, int cls, int entry, int mixture, int bin, int* is_debug)
{
    ctf::set_thread_error("");
#ifdef CTFMNMF_DEBUG
    if (is_debug) *is_debug = 1;
#else
    if (is_debug) *is_debug = 0;
#endif
    if (!b) return fail_b(CTFMNMF_EINVAL, "batch is NULL");
    if (cls < 0 || cls >= (int)b->plan.bins.size()) return fail_b(CTFMNMF_EINVAL, "no such bin class");
    const BatchClass& c = b->plan.bins[cls];
    if (entry < 0 || entry >= c.blocks) return fail_b(CTFMNMF_EINVAL, "no such entry in the bin class");
    if (mixture < 0 || mixture >= (int)b->hs.size()) return fail_b(CTFMNMF_EINVAL, "no such mixture");
#ifdef CTFMNMF_DEBUG
    const int2 w = make_int2(mixture, bin);
    cudaStream_t st = b->hs[0]->stream;
    if (cudaMemcpyAsync(c.work + entry, &w, sizeof(int2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        return fail_b(CTFMNMF_ECUDA, "work-list write failed: %s", cudaGetErrorString(e));
    }
    return CTFMNMF_OK;
#else
    (void)bin;
    return fail_b(CTFMNMF_EUNSUPPORTED, "work lists can be changed only in a CTFMNMF_DEBUG build");
#endif
}

int ctfmnmf_batch_load_stft(ctfmnmf_batch_t b, const void* X, const long long* offsets)
{
    ctf::set_thread_error("");
    if (!b || !X || !offsets) return fail_b(CTFMNMF_EINVAL, "need a batch, a buffer and offsets");
    cudaStream_t st = b->hs[0]->stream;
    for (size_t k = 0; k < b->hs.size(); ++k) {
        ctfmnmf* h = b->hs[k];
        h->loaded = false;
        if (offsets[k] < 0) return fail_b(CTFMNMF_EINVAL, "negative offset");
        const float2* Xk = static_cast<const float2*>(X) + offsets[k];
        if (cudaMemsetAsync(h->d.flag, 0, sizeof(int) * 2, st) != cudaSuccess ||
            ctf::launch_load(h->s, h->d, Xk, st) != cudaSuccess)
            return fail_b(CTFMNMF_ECUDA, "loading a mixture failed");
        if (h->d.X &&
            cudaMemcpyAsync(h->d.X, h->d.Y, sizeof(float2) * (size_t)h->s.F * h->s.M * h->s.Jp,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return fail_b(CTFMNMF_ECUDA, "keeping the observation failed");
        h->launches += 1;
    }
    std::vector<int> flags(b->hs.size(), 0);
    for (size_t k = 0; k < b->hs.size(); ++k)
        if (cudaMemcpyAsync(&flags[k], b->hs[k]->d.flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return fail_b(CTFMNMF_ECUDA, "reading the input checks failed");
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail_b(CTFMNMF_ECUDA, "loading the batch failed");
    for (size_t k = 0; k < b->hs.size(); ++k) {
        if (flags[k] & 1) {
            cudaMemsetAsync(b->hs[k]->d.flag, 0, sizeof(int), st);
            return fail_b(CTFMNMF_ENONFINITE, "a mixture's X holds NaN or Inf");
        }
    }
    for (ctfmnmf* h : b->hs) h->loaded = true;
    return CTFMNMF_OK;
}

int ctfmnmf_batch_set_init(ctfmnmf_batch_t b, const float* T0, const long long* t_offsets, const float* V0,
                           const long long* v_offsets)
{
    ctf::set_thread_error("");
    if (!b || (T0 && !t_offsets) || (V0 && !v_offsets)) return fail_b(CTFMNMF_EINVAL, "need a batch and offsets");
    for (size_t k = 0; k < b->hs.size(); ++k) {
        const int rc = ctfmnmf_set_init(b->hs[k], T0 ? T0 + t_offsets[k] : nullptr, V0 ? V0 + v_offsets[k] : nullptr);
        if (rc != CTFMNMF_OK) return fail_b(rc, "%s", ctfmnmf_last_error(b->hs[k]));
    }
    return CTFMNMF_OK;
}

int ctfmnmf_batch_get_separated(ctfmnmf_batch_t b, void* C, const long long* offsets)
{
    ctf::set_thread_error("");
    if (!b || !C || !offsets) return fail_b(CTFMNMF_EINVAL, "need a batch, a buffer and offsets");
    for (size_t k = 0; k < b->hs.size(); ++k) {
        const int rc = ctfmnmf_get_separated(b->hs[k], static_cast<float2*>(C) + offsets[k]);
        if (rc != CTFMNMF_OK) return fail_b(rc, "%s", ctfmnmf_last_error(b->hs[k]));
    }
    return CTFMNMF_OK;
}

int ctfmnmf_batch_destroy(ctfmnmf_batch_t b)
{
    if (!b) return CTFMNMF_OK;
    if (!b->hs.empty()) cudaStreamSynchronize(b->hs[0]->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    free_plan(b->plan);
    if (b->dmix) cudaFree(b->dmix);
    if (b->capture) cudaStreamDestroy(b->capture);
    release_branches(b);
    delete b;
    return CTFMNMF_OK;
}

}  // extern "C"

namespace ctf {
// The iterations of a batch enqueued on st as plain launches, without the finalize of the
// pending normalisation (the differentiable form applies it itself and records it).
cudaError_t batch_enqueue(ctfmnmf_batch_t b, int n_iter, cudaStream_t st)
{
    return enqueue_batch(b, b->plan, n_iter, st);
}
}  // namespace ctf
