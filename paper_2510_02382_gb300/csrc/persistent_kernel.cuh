// Persistent path: every iteration of one ctfmnmf_iterate call in a single cooperative
// launch. Each CTA holds G groups; group k of CTA b owns bins b*G + k, + G*gridDim, ...
// Per iteration:
//   bin phase (ISS sweep + basis MU of its bins, Sec. III) -> grid barrier ->
//   frame items (activation MU + next PSD, Eq. 18), and the last CTA forms mu in FP64
//   (Eq. 19) as the pending scale -> grid barrier (every CTA then reads the scale).
// When every group owns at most one bin and the shared memory allows, the bin's rows and
// W_i stay in shared memory across iterations ("resident"): Y is read from and written to
// HBM once per call instead of once per iteration.
//
// Grid barrier: an arrival counter and a generation word in global memory. Every wait is
// bounded by a timeout on the global timer; a CTA that times out sets the abort word and
// the timeout status, and every CTA then leaves the kernel at its next barrier.
#pragma once

#include "phases.cuh"

namespace ctf {

constexpr int kPersistThreads = 512;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier: thread 0 of every CTA fences its CTA's writes and adds 1 to an arrival
// counter that is never reset within a launch; the CTA whose arrival completes barrier
// number `epoch` (counter = epoch * gridDim.x) publishes `epoch` in the generation word
// (release), the others poll it with relaxed loads and fence once it has moved. Every
// poll is bounded by the timeout; a CTA whose poll runs out sets the timeout status and
// the abort word, and every CTA leaves at its next barrier. Returns false (uniformly in
// the CTA) on abort. Words: sync[0] abort, sync[1] arrivals, sync[2] generation.
__device__ __forceinline__ bool grid_sync(const State& d, unsigned epoch, unsigned long long timeout_ns,
                                          bool skip_arrival)
{
    __shared__ int s_ok2[2];                          // by epoch parity: no reuse race
    int& s_ok = s_ok2[epoch & 1u];
    unsigned* abort_word = d.sync;
    unsigned* count = d.sync + 1;
    unsigned* gen = d.sync + 2;
    __syncthreads();                                  // all of this CTA's writes precede the arrival
    if (threadIdx.x == 0) {
        int ok = ld_relaxed(abort_word) == 0u;
        if (ok) {
            __threadfence();
            const unsigned arrived = skip_arrival ? 0u : atomicAdd(count, 1u) + 1u;
            if (arrived == epoch * gridDim.x) {
                st_release(gen, epoch);
            } else {
                const unsigned long long t0 = global_ns();
                while (ld_relaxed(gen) < epoch) {
                    if (ld_relaxed(abort_word) != 0u) { ok = 0; break; }
                    if (global_ns() - t0 > timeout_ns) {
                        atomicOr(d.flag + 1, 1);
                        atomicExch(abort_word, 1u);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

struct PersistArgs {
    int n_iter, gt, groups, gsm, res_floats, fc, resident, v_tap0, normalize, skip_cta;
    unsigned long long timeout_ns;
};

template <int M, int FPT, int BB>
__global__ void __launch_bounds__(kPersistThreads, 1)
persistent_kernel(const Shape s, const State d, const PersistArgs pa)
{
    extern __shared__ float4 psm4[];
    __shared__ float s_old[CTFMNMF_MAX_M];
    __shared__ double red_cta[(kPersistThreads / 32) * CTFMNMF_MAX_M];
    // Shared memory: [group 0 work | ... | group G-1 work | group 0 rows | ... ]; the frame
    // phase uses the G work regions as one CTA-wide region.
    const int G = pa.groups, GT = pa.gt;
    const int gi = threadIdx.x / GT;
    const Grp g{(int)threadIdx.x - gi * GT, GT, 1 + gi};
    const Grp cta{(int)threadIdx.x, (int)blockDim.x, 0};
    float* psm = reinterpret_cast<float*>(psm4);
    float* gsm = psm + gi * pa.gsm;
    const int gid = gi * gridDim.x + blockIdx.x, TG = gridDim.x * G;   // bins spread over CTAs first
    const int F = s.F, Jp = s.Jp;
    const int items = (Jp / kFrameTile) * s.N;
    float2* Yres = reinterpret_cast<float2*>(psm + G * pa.gsm + gi * pa.res_floats);   // [M][Jp]
    float2* Wres = Yres + M * Jp;                                                       // [M][M]

    if (threadIdx.x < CTFMNMF_MAX_M) s_old[threadIdx.x] = (int)threadIdx.x < M ? d.scale[threadIdx.x] : 1.f;
    __syncthreads();

    float2 y[M][FPT];
    float2 wcol[M];
    if (pa.resident && gid < F) {
        // copy the bin's rows and W_i into shared memory once (no scale applied here)
        const float2* Yb = d.Y + (size_t)gid * M * Jp;
        for (int e = g.tid; e < M * Jp; e += GT) Yres[e] = __ldcg(Yb + e);
        for (int e = g.tid; e < M * M; e += GT) Wres[e] = __ldcg(d.W + (size_t)gid * M * M + e);
        grp_sync(g);
    }

    bool alive = true;
    for (int it = 0; it < pa.n_iter && alive; ++it) {
        // ---- bin phase
        for (int i = gid; i < F; i += TG) {
            float2* Yb = d.Y + (size_t)i * M * Jp;
            float2* Wb = d.W + (size_t)i * M * M;
            float detf;
            if (pa.resident) {
                load_bin<M, FPT, false>(Jp, Yres, Wres, g, s_old, y, wcol);
                detf = bin_body<M, FPT, false, (BB < 16 ? BB : 16)>(s, d, i, g, gsm, y, wcol, Yres, Wres, s_old, pa.v_tap0);
            } else {
                load_bin<M, FPT, true>(Jp, Yb, Wb, g, s_old, y, wcol);
                detf = bin_body<M, FPT, true, (BB < 16 ? BB : 16)>(s, d, i, g, gsm, y, wcol, Yb, Wb, s_old, pa.v_tap0);
            }
            if (g.tid == 0) {
                double f = (double)detf;
#pragma unroll
                for (int r = 0; r < M; ++r) f *= (double)s_old[r];
                logdet_mul(d, i, f);
            }
        }
        alive = grid_sync(d, 2u * it + 1u, pa.timeout_ns, it == 0 && (int)blockIdx.x == pa.skip_cta);
        if (!alive) break;
        // ---- frame items; the last CTA also forms the normalisation scale (FP64) into d.scale
        for (int item = blockIdx.x; item < items; item += gridDim.x) {
            // two frames per thread where the registers allow it (128 per thread here)
            if constexpr (BB <= 10) frame_item<BB>(s, d, item, cta, psm, pa.fc, pa.v_tap0);
            else frame_item_wide<BB>(s, d, item, cta, psm, pa.fc, pa.v_tap0);
        }
        if (blockIdx.x == gridDim.x - 1) {
            scales_fp64<false>(s, d, pa.normalize, red_cta);
            __syncthreads();
        }
        alive = grid_sync(d, 2u * it + 2u, pa.timeout_ns, false);
        if (threadIdx.x < CTFMNMF_MAX_M) s_old[threadIdx.x] = (int)threadIdx.x < M ? __ldcg(d.scale + threadIdx.x) : 1.f;
        __syncthreads();
    }
    if (!alive) return;
    if (pa.resident && gid < F) {
        grp_sync(g);
        float2* Yb = d.Y + (size_t)gid * M * Jp;
        for (int e = g.tid; e < M * Jp; e += GT) __stcg(Yb + e, Yres[e]);
        for (int e = g.tid; e < M * M; e += GT) __stcg(d.W + (size_t)gid * M * M + e, Wres[e]);
    }
}

// Per-M instantiation tables (persistent_m*.cu), compiled as separate translation units.
const void* persistent_ptr_m2(int BB);
const void* persistent_ptr_m3(int BB);
const void* persistent_ptr_m4(int BB);
const void* persistent_ptr_m5(int BB);
const void* persistent_ptr_m6(int BB);
const void* persistent_ptr_m7(int BB);
const void* persistent_ptr_m8(int BB);

}  // namespace ctf
