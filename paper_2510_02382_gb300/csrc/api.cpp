// Host side of the C ABI declared in include/ctfmnmf.h: argument checks, device
// buffers, the launch sequence of one call and the CUDA-graph cache of ctfmnmf_iterate.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "handle.h"

namespace {

thread_local char g_create_err[256] = "";

int fail(ctfmnmf* h, int code, const char* fmt, ...)
{
    char* buf = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(h, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail((h), CTFMNMF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

void free_state(ctfmnmf* h)
{
    State& d = h->d;
    void* ptrs[] = {d.Y, d.W, d.logdet, d.T, d.V, d.invlam, d.P, d.mupart, d.scale, d.flag,
                    d.cost_part, d.cost_out, d.staging, d.detb, d.ldm, d.lde, d.sync, d.X};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    memset(&h->d, 0, sizeof(h->d));
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    if (h->capture) cudaStreamDestroy(h->capture);
    h->capture = nullptr;
    if (h->host_cost) cudaFreeHost(h->host_cost);
    h->host_cost = nullptr;
    if (h->sepbuf) cudaFree(h->sepbuf);
    h->sepbuf = nullptr;
}

int check_flag(ctfmnmf* h, int mask, const char* what)
{
    int flag = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&flag, h->d.flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (flag & mask) {
        CUDA_TRY(h, cudaMemsetAsync(h->d.flag, 0, sizeof(int), h->stream));
        return fail(h, CTFMNMF_ENONFINITE, "%s holds NaN or Inf", what);
    }
    return CTFMNMF_OK;
}

using ctf::kFinalizeKernels;

// Synchronise the stream and report what the device recorded since the last report (then
// clear it): flag[1] a bounded wait ran out, flag[2] the NaN/Inf scan found a non-finite value,
// flag[3] a bounds check of a debug build stopped a block. The state is unusable after any.
int sync_and_check(ctfmnmf* h)
{
    int flag[3] = {0, 0, 0};
    CUDA_TRY(h, cudaMemcpyAsync(flag, h->d.flag + 1, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (flag[0] || flag[1] || flag[2]) {
        CUDA_TRY(h, cudaMemsetAsync(h->d.flag + 1, 0, 3 * sizeof(int), h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        h->loaded = false;
        if (flag[2]) return fail(h, CTFMNMF_EBOUNDS, "a device-side bounds check stopped a thread block");
        if (flag[0]) return fail(h, CTFMNMF_ETIMEOUT, "a device-side wait of the persistent kernel ran out");
        return fail(h, CTFMNMF_ENONFINITE, "the state holds NaN or Inf after an iteration");
    }
    return CTFMNMF_OK;
}

int enqueue_iterations(ctfmnmf* h, int n_iter, cudaStream_t st)
{
    const int tap0 = h->opt.v_update == CTFMNMF_V_TAP0;
    const bool ip = h->opt.w_update == CTFMNMF_W_IP;
    for (int t = 0; t < n_iter; ++t) {
        CUDA_TRY(h, ip ? ctf::launch_ip_bin_phase(h->s, h->d, tap0, st)
                       : h->cplan.ok ? ctf::launch_cluster_bin_phase(h->s, h->d, tap0, h->cplan, st)
                                     : ctf::launch_bin_phase_as(h->s, h->d, tap0, h->bin_fpt, h->bin_nt, st));
        CUDA_TRY(h, ctf::launch_frame_phase(h->s, h->d, tap0, h->opt.normalize, st));
        if (h->opt.check_finite) CUDA_TRY(h, ctf::launch_finite_scan(h->s, h->d, st));
    }
    CUDA_TRY(h, ctf::launch_finalize(h->s, h->d, st));
    return CTFMNMF_OK;
}

}  // namespace

long long ctf::iteration_kernels(int n_iter, bool scan) { return (scan ? 3LL : 2LL) * n_iter + kFinalizeKernels; }

namespace {
using ctf::iteration_kernels;

}  // namespace

void ctf::set_thread_error(const char* msg)
{
    snprintf(g_create_err, sizeof(g_create_err), "%s", msg);
}

extern "C" {

void ctfmnmf_default_options(ctfmnmf_options* opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->v_update = CTFMNMF_V_ALL_TAPS;
    opt->normalize = 1;
    opt->use_graph = 1;
    opt->deterministic_reduce = 1;
}

// AUTO: time a few iterations of each candidate on a probe state and keep the fastest — the
// persistent kernel (when it fits) and the two-kernel path with each bin-phase shape
// (frames per thread, threads). Neither path nor shape wins for every mixture: launch gaps
// against grid barriers and register budgets, block-level reductions against per-thread
// work. Then return the handle to the state of a fresh one (default factors, nothing
// loaded). Synchronous, a few milliseconds; on any failure the defaults stay.
static void choose_path(ctfmnmf* h)
{
    constexpr int kIters = 3;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // candidates: the persistent kernel, then the two-kernel path with each bin-phase shape
    int fpts[5] = {0, 0, 0, 0, 0}, nts[5] = {0, 0, 0, 0, 0};
    int nc = ctf::bin_phase_candidates(h->s.M, h->s.J, fpts, nts);
    if (ctf::contig_supported(h->s)) {                 // eight contiguous frames per thread
        fpts[nc] = ctf::kBinContig;
        nts[nc] = ctf::contig_threads(h->s);
        ++nc;
    }
    const int def_fpt = h->bin_fpt, def_nt = h->bin_nt;
    if (h->opt.bin_fpt != 0) {                          // a forced shape is the only candidate
        fpts[0] = def_fpt;
        nts[0] = def_nt;
        nc = 1;
    }
    float best = 1e30f;
    int best_c = -2;                                    // -1: persistent, >= 0: candidate, -2: none
    bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
              ctf::launch_probe_fill(h->s, h->d, h->stream) == cudaSuccess;
    h->loaded = true;
    for (int c = h->plan.ok ? -1 : 0; c < nc && ok; ++c) {
        if (c >= 0 && (ctf::configure_bin_phase_as(h->s, fpts[c], nts[c]) != cudaSuccess)) {
            cudaGetLastError();
            continue;
        }
        h->path = c < 0 ? CTFMNMF_PATH_PERSISTENT : CTFMNMF_PATH_TWO_KERNEL;
        if (c >= 0) {
            h->bin_fpt = fpts[c];
            h->bin_nt = nts[c];
        }
        if (h->graph) {                                 // the graph holds the bin-phase shape
            cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
        }
        float ms = 0.f;
        ok = ctfmnmf_iterate(h, kIters) == CTFMNMF_OK &&                 // warm-up (and graph capture)
             cudaEventRecord(e0, h->stream) == cudaSuccess && ctfmnmf_iterate(h, kIters) == CTFMNMF_OK &&
             cudaEventRecord(e1, h->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok && ms < best) {
            best = ms;
            best_c = c;
        }
    }
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->path = best_c >= 0 ? CTFMNMF_PATH_TWO_KERNEL : CTFMNMF_PATH_PERSISTENT;
    h->bin_fpt = best_c >= 0 ? fpts[best_c] : def_fpt;
    h->bin_nt = best_c >= 0 ? nts[best_c] : def_nt;
    if (!ok || best_c == -2) {                          // nothing timed: the defaults
        h->path = h->plan.ok ? CTFMNMF_PATH_PERSISTENT : CTFMNMF_PATH_TWO_KERNEL;
        h->bin_fpt = def_fpt;
        h->bin_nt = def_nt;
    }
    h->loaded = false;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ctf::launch_init_nmf(h->s, h->d, nullptr, nullptr, 0, h->stream);
    ctf::launch_psd(h->s, h->d, h->stream);
    cudaStreamSynchronize(h->stream);
    cudaGetLastError();
    h->err[0] = 0;
    h->launches = 0;
}

int ctfmnmf_create(int M, int N, int L, int B, int F, int J, ctfmnmf_t* out)
{
    ctfmnmf_dims d = {M, N, L, B, F, J};
    return ctfmnmf_create_ex(&d, nullptr, nullptr, out);
}

int ctfmnmf_create_ex(const ctfmnmf_dims* dims, const int* Ln, const ctfmnmf_options* opt,
                      ctfmnmf_t* out)
{
    g_create_err[0] = 0;
    if (!out) return fail(nullptr, CTFMNMF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!dims) return fail(nullptr, CTFMNMF_EINVAL, "dims is NULL");
    const int M = dims->M, N = dims->N, L = dims->L, B = dims->B, F = dims->F, J = dims->J;
    if (M <= 0 || N <= 0 || L <= 0 || B <= 0 || F <= 0 || J <= 0)
        return fail(nullptr, CTFMNMF_EINVAL, "every dimension must be positive");
    if (N > M) return fail(nullptr, CTFMNMF_EINVAL, "N=%d sources exceed M=%d microphones", N, M);
    if (M > CTFMNMF_MAX_M) return fail(nullptr, CTFMNMF_EINVAL, "M=%d exceeds %d", M, CTFMNMF_MAX_M);
    if (B > CTFMNMF_MAX_B) return fail(nullptr, CTFMNMF_EINVAL, "B=%d exceeds %d", B, CTFMNMF_MAX_B);
    ctfmnmf_options o;
    ctfmnmf_default_options(&o);
    if (opt) {
        o = *opt;
        if (o.v_update != CTFMNMF_V_ALL_TAPS && o.v_update != CTFMNMF_V_TAP0)
            return fail(nullptr, CTFMNMF_EINVAL, "unknown v_update %d", o.v_update);
        if ((o.normalize != 0 && o.normalize != 1) || (o.use_graph != 0 && o.use_graph != 1))
            return fail(nullptr, CTFMNMF_EINVAL, "normalize and use_graph must be 0 or 1");
        if (o.path < CTFMNMF_PATH_AUTO || o.path > CTFMNMF_PATH_PERSISTENT)
            return fail(nullptr, CTFMNMF_EINVAL, "unknown path %d", o.path);
        if (o.wait_timeout_ms < 0) return fail(nullptr, CTFMNMF_EINVAL, "wait_timeout_ms must be >= 0");
        if (o.w_update != CTFMNMF_W_ISS && o.w_update != CTFMNMF_W_IP)
            return fail(nullptr, CTFMNMF_EINVAL, "unknown w_update %d", o.w_update);
        if (o.reserved[0]) return fail(nullptr, CTFMNMF_EINVAL, "reserved options must be 0");
        if (o.bin_fpt != 0 && o.bin_fpt != 1 && o.bin_fpt != 2 && o.bin_fpt != 4 && o.bin_fpt != 8 &&
            o.bin_fpt != ctf::kBinContig)
            return fail(nullptr, CTFMNMF_EINVAL, "bin_fpt must be 0, 1, 2, 4, 8 or -8");
        if (!(o.eps_floor >= 0.f) || !(o.eps_floor < 3.0e38f))
            return fail(nullptr, CTFMNMF_EINVAL, "eps_floor must be finite and >= 0");
        if ((o.deterministic_reduce != 0 && o.deterministic_reduce != 1) || (o.check_finite != 0 && o.check_finite != 1))
            return fail(nullptr, CTFMNMF_EINVAL, "deterministic_reduce and check_finite must be 0 or 1");
    }
#ifdef CTFMNMF_DEBUG
    o.check_finite = 1;                            // debug builds always scan for NaN/Inf
#endif
    Shape s;
    memset(&s, 0, sizeof(s));
    s.M = M; s.N = N; s.B = B; s.F = F; s.J = J;
    s.Jp = (J + 7) / 8 * 8;
    s.FBp = (F * B + 3) / 4 * 4;
    s.invJ = 1.0 / (double)J;
    s.floor_nmf = o.eps_floor > 0.f ? o.eps_floor : ctf::kFloorNmf;
    s.det_reduce = o.deterministic_reduce;
    int total = 0, lmax = 0;
    for (int n = 0; n < N; ++n) {
        const int t = Ln ? Ln[n] : M / N + (n < M % N ? 1 : 0);
        if (t <= 0) return fail(nullptr, CTFMNMF_EINVAL, "tap count of source %d must be positive", n);
        if (t > L) return fail(nullptr, CTFMNMF_EINVAL, "source %d has %d taps, more than L=%d", n, t, L);
        s.Ln[n] = t;
        s.row0[n] = total;
        for (int l = 0; l < t && total + l < CTFMNMF_MAX_M; ++l) {
            s.row_n[total + l] = n;
            s.row_l[total + l] = l;
        }
        total += t;
        if (t > lmax) lmax = t;
    }
    if (total != M) return fail(nullptr, CTFMNMF_EINVAL, "taps sum to %d, not M=%d", total, M);
    if (J <= lmax) return fail(nullptr, CTFMNMF_EINVAL, "J=%d frames must exceed the longest tap count %d", J, lmax);
    int fpt = 0, nt = 0;
    const bool one_block = ctf::bin_phase_config(M, J, &fpt, &nt);
    if (!one_block && J > ctf::cluster_max_frames(M))
        return fail(nullptr, CTFMNMF_EUNSUPPORTED, "J=%d frames is too long for M=%d (at most %d)", J, M,
                    ctf::cluster_max_frames(M));
    if (o.bin_fpt == ctf::kBinContig) {            // eight contiguous frames per thread, default taps
        if (!ctf::contig_supported(s))
            return fail(nullptr, CTFMNMF_EUNSUPPORTED, "bin_fpt=-8 needs M <= 4, the default taps and J <= 4096");
        fpt = ctf::kBinContig;
        nt = ctf::contig_threads(s);
    } else if (o.bin_fpt != 0) {                   // a forced bin-phase shape must be a candidate
        int fpts[4], nts[4];
        const int nc = ctf::bin_phase_candidates(M, J, fpts, nts);
        int k = 0;
        while (k < nc && fpts[k] != o.bin_fpt) ++k;
        if (k == nc)
            return fail(nullptr, CTFMNMF_EUNSUPPORTED, "bin_fpt=%d cannot run J=%d frames with M=%d", o.bin_fpt, J, M);
        fpt = fpts[k];
        nt = nts[k];
    }
    const bool ip = o.w_update == CTFMNMF_W_IP;
    if (ip && !one_block)
        return fail(nullptr, CTFMNMF_EUNSUPPORTED, "the IP update needs a bin's frames in one thread block");
    if (ip && M > 4) return fail(nullptr, CTFMNMF_EUNSUPPORTED, "the IP update supports M <= 4 (M=%d)", M);
    if (ip && o.path == CTFMNMF_PATH_PERSISTENT)
        return fail(nullptr, CTFMNMF_EUNSUPPORTED, "the IP update runs on the two-kernel path only");

    ctfmnmf* h = new (std::nothrow) ctfmnmf;
    if (!h) return fail(nullptr, CTFMNMF_ENOMEM, "host allocation failed");
    memset(h, 0, sizeof(*h));
    h->s = s;
    h->opt = o;
    h->L = L;
    cudaGetDevice(&h->device);

    State& d = h->d;
    const size_t MF = (size_t)M * F, FNJ = (size_t)F * N * s.Jp;
    struct { void** p; size_t bytes; } allocs[] = {
        {(void**)&d.Y, sizeof(float2) * MF * s.Jp},
        {(void**)&d.W, sizeof(float2) * MF * M},
        {(void**)&d.logdet, sizeof(double) * F},
        {(void**)&d.T, sizeof(float) * (size_t)N * s.FBp},
        {(void**)&d.V, sizeof(float) * (size_t)N * B * s.Jp},
        {(void**)&d.invlam, sizeof(float) * FNJ},
        {(void**)&d.P, sizeof(float) * FNJ},
        {(void**)&d.mupart, sizeof(double) * MF},
        {(void**)&d.scale, sizeof(float) * CTFMNMF_MAX_M},
        {(void**)&d.flag, sizeof(int) * 4},
        {(void**)&d.cost_part, sizeof(double) * F},
        {(void**)&d.cost_out, sizeof(double)},
        {(void**)&d.detb, sizeof(float) * F},
        {(void**)&d.ldm, sizeof(double) * F},
        {(void**)&d.lde, sizeof(int) * F},
        {(void**)&d.sync, sizeof(unsigned) * 32},
        {(void**)&d.X, ip ? sizeof(float2) * MF * s.Jp : 0},
    };
    for (auto& a : allocs) {
        if (a.bytes == 0) continue;
        if (cudaMalloc(a.p, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            free_state(h);
            delete h;
            return fail(nullptr, CTFMNMF_ENOMEM, "cudaMalloc of %zu bytes failed", a.bytes);
        }
    }
    int rc = CTFMNMF_OK;
    if (cudaMallocHost((void**)&h->host_cost, sizeof(double)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking) != cudaSuccess) {
        rc = CTFMNMF_ECUDA;
    }
    if (rc == CTFMNMF_OK && (cudaMemset(d.flag, 0, sizeof(int) * 4) != cudaSuccess ||
                             cudaMemset(d.sync, 0, sizeof(unsigned) * 32) != cudaSuccess ||
                             cudaMemset(d.P, 0, sizeof(float) * FNJ) != cudaSuccess ||
                             cudaMemset(d.mupart, 0, sizeof(double) * MF) != cudaSuccess))
        rc = CTFMNMF_ECUDA;
    if (rc == CTFMNMF_OK && !one_block) {
        h->cplan = ctf::plan_cluster(s);
        if (!h->cplan.ok) {
            free_state(h);
            delete h;
            return fail(nullptr, CTFMNMF_EUNSUPPORTED, "J=%d frames do not fit a cluster of 8 blocks on this device", J);
        }
    }
    if (rc == CTFMNMF_OK && ip && ctf::configure_ip_bin_phase(s) != cudaSuccess) rc = CTFMNMF_ECUDA;
    if (rc == CTFMNMF_OK && (h->cplan.ok ? ctf::configure_cluster_bin_phase(s, h->cplan)
                                         : ctf::configure_bin_phase_as(s, fpt, nt)) != cudaSuccess)
        rc = CTFMNMF_ECUDA;
    if (rc == CTFMNMF_OK && (
                             ctf::configure_frame_phase() != cudaSuccess ||
                             ctf::launch_init_nmf(s, d, nullptr, nullptr, 0, nullptr) != cudaSuccess ||
                             ctf::launch_psd(s, d, nullptr) != cudaSuccess ||
                             cudaDeviceSynchronize() != cudaSuccess))
        rc = CTFMNMF_ECUDA;
    if (rc != CTFMNMF_OK) {
        const char* msg = cudaGetErrorString(cudaGetLastError());
        free_state(h);
        delete h;
        return fail(nullptr, rc, "device set-up failed: %s", msg);
    }
    h->bin_fpt = one_block ? fpt : 0;
    h->bin_nt = one_block ? nt : 0;
    h->skip_cta = -1;
    h->timeout_ns = 1000000ull * (unsigned long long)(o.wait_timeout_ms > 0 ? o.wait_timeout_ms : 2000);
    if (!ip) h->plan = ctf::plan_persistent(s);
    cudaGetLastError();
    if (o.path == CTFMNMF_PATH_PERSISTENT && !h->plan.ok) {
        free_state(h);
        delete h;
        return fail(nullptr, CTFMNMF_EUNSUPPORTED, "the persistent path does not fit this shape on this device");
    }
    h->path = (o.path != CTFMNMF_PATH_TWO_KERNEL && h->plan.ok) ? CTFMNMF_PATH_PERSISTENT
                                                                 : CTFMNMF_PATH_TWO_KERNEL;
    if (o.path == CTFMNMF_PATH_AUTO && !ip && !h->cplan.ok) choose_path(h);
    *out = h;
    return CTFMNMF_OK;
}

int ctfmnmf_destroy(ctfmnmf_t h)
{
    if (!h) return CTFMNMF_OK;
    cudaStreamSynchronize(h->stream);
    free_state(h);
    delete h;
    return CTFMNMF_OK;
}

const char* ctfmnmf_last_error(ctfmnmf_t h) { return h ? h->err : g_create_err; }

int ctfmnmf_set_stream(ctfmnmf_t h, void* stream)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    h->stream = (cudaStream_t)stream;
    return CTFMNMF_OK;
}

int ctfmnmf_get_taps(ctfmnmf_t h, int* Ln)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!Ln) return fail(h, CTFMNMF_EINVAL, "Ln is NULL");
    for (int n = 0; n < h->s.N; ++n) Ln[n] = h->s.Ln[n];
    return CTFMNMF_OK;
}

int ctfmnmf_load_stft(ctfmnmf_t h, const void* X)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!X) return fail(h, CTFMNMF_EINVAL, "X is NULL");
    h->err[0] = 0;
    h->loaded = false;
    CUDA_TRY(h, cudaMemsetAsync(h->d.flag + 1, 0, sizeof(int), h->stream));
    CUDA_TRY(h, ctf::launch_load(h->s, h->d, (const float2*)X, h->stream));
    CUDA_TRY(h, ctf::launch_psd(h->s, h->d, h->stream));
    h->launches += 2;
    if (h->d.X)       // the IP update demixes the observation itself: keep it (bin-major, padded)
        CUDA_TRY(h, cudaMemcpyAsync(h->d.X, h->d.Y, sizeof(float2) * (size_t)h->s.F * h->s.M * h->s.Jp,
                                    cudaMemcpyDeviceToDevice, h->stream));
    int rc = check_flag(h, 1, "X");
    if (rc != CTFMNMF_OK) return rc;
    h->loaded = true;
    return CTFMNMF_OK;
}

int ctfmnmf_load_stft_host(ctfmnmf_t h, const void* X)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!X) return fail(h, CTFMNMF_EINVAL, "X is NULL");
    const size_t bytes = sizeof(float2) * (size_t)h->s.M * h->s.F * h->s.J;
    if (!h->d.staging) {
        if (cudaMalloc((void**)&h->d.staging, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, CTFMNMF_ENOMEM, "cudaMalloc of %zu staging bytes failed", bytes);
        }
    }
    CUDA_TRY(h, cudaMemcpyAsync(h->d.staging, X, bytes, cudaMemcpyHostToDevice, h->stream));
    return ctfmnmf_load_stft(h, h->d.staging);
}

int ctfmnmf_set_state(ctfmnmf_t h, const void* Y, const void* W, const float* T, const float* V,
                      const double* logdet)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!Y || !W || !T || !V || !logdet) return fail(h, CTFMNMF_EINVAL, "null pointer argument");
    if (h->d.X && !h->loaded) return fail(h, CTFMNMF_ESTATE, "the IP update needs ctfmnmf_load_stft first");
    h->err[0] = 0;
    h->loaded = false;
    const Shape& s = h->s;
    // the rows in the loaded layout (as ctfmnmf_load_stft does with X; it also resets W,
    // log|det| and the pending scale), then W, log|det| and the factors over them
    CUDA_TRY(h, ctf::launch_load(s, h->d, (const float2*)Y, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->d.W, W, sizeof(float2) * (size_t)s.F * s.M * s.M, cudaMemcpyDeviceToDevice,
                                h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->d.logdet, logdet, sizeof(double) * s.F, cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(h, ctf::launch_init_nmf(s, h->d, T, V, 0, h->stream));
    CUDA_TRY(h, ctf::launch_psd(s, h->d, h->stream));
    h->launches += 3;
    int rc = check_flag(h, 3, "the state");
    if (rc != CTFMNMF_OK) return rc;
    h->loaded = true;
    return CTFMNMF_OK;
}

int ctfmnmf_set_init(ctfmnmf_t h, const float* T0, const float* V0)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    h->err[0] = 0;
    if (!T0 && !V0) return CTFMNMF_OK;
    CUDA_TRY(h, ctf::launch_init_nmf(h->s, h->d, T0, V0, 0, h->stream));
    CUDA_TRY(h, ctf::launch_psd(h->s, h->d, h->stream));
    h->launches += 2;
    return check_flag(h, 2, "T0/V0");
}

int ctfmnmf_iterate(ctfmnmf_t h, int n_iter)
{
    ctf::TraceRange trace("ctfmnmf_iterate");
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (n_iter < 0) return fail(h, CTFMNMF_EINVAL, "n_iter=%d is negative", n_iter);
    if (!h->loaded) return fail(h, CTFMNMF_ESTATE, "no STFT loaded");
    h->err[0] = 0;
    if (n_iter == 0) return CTFMNMF_OK;
    if (h->path == CTFMNMF_PATH_PERSISTENT) {
        const int tap0 = h->opt.v_update == CTFMNMF_V_TAP0;
        CUDA_TRY(h, ctf::launch_persistent(h->s, h->d, h->plan, n_iter, tap0, h->opt.normalize, h->timeout_ns,
                                           h->skip_cta, h->stream));
        h->skip_cta = -1;
        CUDA_TRY(h, ctf::launch_finalize(h->s, h->d, h->stream));
        h->launches += 1 + kFinalizeKernels;
        if (h->opt.check_finite) {
            CUDA_TRY(h, ctf::launch_finite_scan(h->s, h->d, h->stream));
            h->launches += 1;
        }
        return CTFMNMF_OK;
    }
    if (!h->opt.use_graph) {
        const int rc = enqueue_iterations(h, n_iter, h->stream);
        if (rc == CTFMNMF_OK) h->launches += iteration_kernels(n_iter, h->opt.check_finite != 0);
        return rc;
    }
    if (!h->graph || h->graph_iters != n_iter) {
        if (h->graph) {
            cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        CUDA_TRY(h, cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_iterations(h, n_iter, h->capture);
        cudaError_t ec = cudaStreamEndCapture(h->capture, &g);
        if (rc != CTFMNMF_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) return fail(h, CTFMNMF_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
        ec = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (ec != cudaSuccess) {
            h->graph = nullptr;
            return fail(h, CTFMNMF_ECUDA, "graph instantiate: %s", cudaGetErrorString(ec));
        }
        h->graph_iters = n_iter;
    }
    CUDA_TRY(h, cudaGraphLaunch(h->graph, h->stream));
    h->launches += iteration_kernels(n_iter, h->opt.check_finite != 0);
    return CTFMNMF_OK;
}

int ctfmnmf_cost(ctfmnmf_t h, double* out)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!out) return fail(h, CTFMNMF_EINVAL, "out is NULL");
    if (!h->loaded) return fail(h, CTFMNMF_ESTATE, "no STFT loaded");
    {
        const int rc = sync_and_check(h);
        if (rc != CTFMNMF_OK) return rc;
    }
    CUDA_TRY(h, ctf::launch_cost(h->s, h->d, h->stream));
    h->launches += 2;
    CUDA_TRY(h, cudaMemcpyAsync(h->host_cost, h->d.cost_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    *out = *h->host_cost;
    return CTFMNMF_OK;
}

int ctfmnmf_get_separated(ctfmnmf_t h, void* C)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!C) return fail(h, CTFMNMF_EINVAL, "output is NULL");
    if (!h->loaded) return fail(h, CTFMNMF_ESTATE, "no STFT loaded");
    CUDA_TRY(h, ctf::launch_separate(h->s, h->d, (float2*)C, h->stream));
    h->launches += 1;
    return CTFMNMF_OK;
}

int ctfmnmf_get_separated_host(ctfmnmf_t h, void* C)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!C) return fail(h, CTFMNMF_EINVAL, "output is NULL");
    if (!h->loaded) return fail(h, CTFMNMF_ESTATE, "no STFT loaded");
    const size_t bytes = sizeof(float2) * (size_t)h->s.N * h->s.M * h->s.F * h->s.J;
    if (!h->sepbuf) {
        if (cudaMalloc((void**)&h->sepbuf, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, CTFMNMF_ENOMEM, "cudaMalloc of %zu output bytes failed", bytes);
        }
    }
    CUDA_TRY(h, ctf::launch_separate(h->s, h->d, h->sepbuf, h->stream));
    h->launches += 1;
    CUDA_TRY(h, cudaMemcpyAsync(C, h->sepbuf, bytes, cudaMemcpyDeviceToHost, h->stream));
    {
        const int rc = sync_and_check(h);
        if (rc != CTFMNMF_OK) return rc;
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return CTFMNMF_OK;
}

int ctfmnmf_get_demixed(ctfmnmf_t h, void* Y)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!Y) return fail(h, CTFMNMF_EINVAL, "output is NULL");
    CUDA_TRY(h, ctf::launch_get_demixed(h->s, h->d, (float2*)Y, h->stream));
    h->launches += 1;
    return CTFMNMF_OK;
}

int ctfmnmf_get_demix_matrix(ctfmnmf_t h, void* W)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!W) return fail(h, CTFMNMF_EINVAL, "output is NULL");
    CUDA_TRY(h, cudaMemcpyAsync(W, h->d.W, sizeof(float2) * (size_t)h->s.F * h->s.M * h->s.M,
                                cudaMemcpyDeviceToDevice, h->stream));
    return CTFMNMF_OK;
}

int ctfmnmf_get_logdet(ctfmnmf_t h, double* logdet)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!logdet) return fail(h, CTFMNMF_EINVAL, "output is NULL");
    CUDA_TRY(h, cudaMemcpyAsync(logdet, h->d.logdet, sizeof(double) * h->s.F, cudaMemcpyDeviceToDevice,
                                h->stream));
    return CTFMNMF_OK;
}

int ctfmnmf_get_nmf(ctfmnmf_t h, float* T, float* V)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!T && !V) return CTFMNMF_OK;
    CUDA_TRY(h, ctf::launch_get_nmf(h->s, h->d, T, V, h->stream));
    h->launches += 1;
    return CTFMNMF_OK;
}

int ctfmnmf_time_phases(ctfmnmf_t h, int n_iter, double* ms)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!ms || n_iter < 1) return fail(h, CTFMNMF_EINVAL, "need n_iter >= 1 and an output");
    if (!h->loaded) return fail(h, CTFMNMF_ESTATE, "no STFT loaded");
    const int tap0 = h->opt.v_update == CTFMNMF_V_TAP0;
    cudaEvent_t ev[4];
    for (auto& e : ev) CUDA_TRY(h, cudaEventCreate(&e));
    double tot[2] = {0.0, 0.0};
    int rc = CTFMNMF_OK;
    for (int t = 0; t < n_iter && rc == CTFMNMF_OK; ++t) {
        cudaError_t e = cudaEventRecord(ev[0], h->stream);
        if (e == cudaSuccess)
            e = h->opt.w_update == CTFMNMF_W_IP ? ctf::launch_ip_bin_phase(h->s, h->d, tap0, h->stream)
                : h->cplan.ok ? ctf::launch_cluster_bin_phase(h->s, h->d, tap0, h->cplan, h->stream)
                              : ctf::launch_bin_phase_as(h->s, h->d, tap0, h->bin_fpt, h->bin_nt, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], h->stream);
        if (e == cudaSuccess) e = ctf::launch_frame_phase(h->s, h->d, tap0, h->opt.normalize, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3], h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
        float a = 0.f, b = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[2], ev[3]);
        if (e != cudaSuccess) rc = fail(h, CTFMNMF_ECUDA, "phase timing: %s", cudaGetErrorString(e));
        tot[0] += a;
        tot[1] += b;
    }
    if (rc == CTFMNMF_OK && ctf::launch_finalize(h->s, h->d, h->stream) != cudaSuccess)
        rc = fail(h, CTFMNMF_ECUDA, "finalize launch failed");
    if (rc == CTFMNMF_OK) h->launches += iteration_kernels(n_iter, false);
    for (auto& e : ev) cudaEventDestroy(e);
    if (rc != CTFMNMF_OK) return rc;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    ms[0] = tot[0] / n_iter;
    ms[1] = tot[1] / n_iter;
    return CTFMNMF_OK;
}

int ctfmnmf_synchronize(ctfmnmf_t h)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    return sync_and_check(h);
}

int ctfmnmf_get_path(ctfmnmf_t h, int* path)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!path) return fail(h, CTFMNMF_EINVAL, "path is NULL");
    *path = h->path;
    return CTFMNMF_OK;
}

int ctfmnmf_get_bin_shape(ctfmnmf_t h, int* fpt, int* threads)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!fpt || !threads) return fail(h, CTFMNMF_EINVAL, "need two outputs");
    *fpt = h->cplan.ok ? 0 : h->bin_fpt;
    *threads = h->cplan.ok ? 0 : h->bin_nt;
    return CTFMNMF_OK;
}

int ctfmnmf_time_persistent(ctfmnmf_t h, int n_iter, double* ms)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!ms || n_iter < 1) return fail(h, CTFMNMF_EINVAL, "need n_iter >= 1 and an output");
    if (!h->loaded) return fail(h, CTFMNMF_ESTATE, "no STFT loaded");
    if (h->path != CTFMNMF_PATH_PERSISTENT) return fail(h, CTFMNMF_EUNSUPPORTED, "handle uses the two-kernel path");
    const int tap0 = h->opt.v_update == CTFMNMF_V_TAP0;
    cudaEvent_t ev[4];
    for (auto& e : ev) CUDA_TRY(h, cudaEventCreate(&e));
    cudaError_t e = cudaEventRecord(ev[0], h->stream);
    if (e == cudaSuccess)
        e = ctf::launch_persistent(h->s, h->d, h->plan, n_iter, tap0, h->opt.normalize, h->timeout_ns, -1,
                                   h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], h->stream);
    if (e == cudaSuccess) e = ctf::launch_finalize(h->s, h->d, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
    float a = 0.f, b = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[2], ev[3]);
    for (auto& x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return fail(h, CTFMNMF_ECUDA, "persistent timing: %s", cudaGetErrorString(e));
    h->launches += 1 + kFinalizeKernels;
    const int rc = sync_and_check(h);
    if (rc != CTFMNMF_OK) return rc;
    ms[0] = a;
    ms[1] = b;
    return CTFMNMF_OK;
}

int ctfmnmf_debug_skip_arrival(ctfmnmf_t h, int cta)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (cta >= 0 && h->path != CTFMNMF_PATH_PERSISTENT)
        return fail(h, CTFMNMF_EUNSUPPORTED, "handle uses the two-kernel path");
    h->skip_cta = cta < 0 ? -1 : cta;
    return CTFMNMF_OK;
}

int ctfmnmf_get_launch_count(ctfmnmf_t h, long long* count)
{
    if (!h) return fail(nullptr, CTFMNMF_EINVAL, "handle is NULL");
    if (!count) return fail(h, CTFMNMF_EINVAL, "count is NULL");
    *count = h->launches;
    return CTFMNMF_OK;
}

}  // extern "C"
