// Bin phase with contiguous frames per thread and a compile-time tap layout (one CTF-MNMF-ISS
// bin update of Sec. III: ISS sweep of Eqs. 11-16, row powers of Eq. 19, delayed power, basis
// MU of Eq. 17), used for M <= 4 with the default taps L_n = floor(M/N) + (n < M mod N).
//
// Thread t of the block owns the 8 frames j0 = 8t .. 8t+7 of the bin, so
//   * its rows load and store as 16-byte vectors (two complex64 per access),
//   * the delayed weights phi_r(j) = 1/lambda_{n(r)}(j - l(r)) of its frames are one aligned
//     16-float window of the staged 1/lambda per source, from which every tap's shift is a
//     compile-time register choice,
//   * the delayed power P_n(j) = sum_l |y_{(n,l)}(j + l)|^2 needs, besides its own frames,
//     only the first L_n - 1 frames of the next thread (one shuffle per delayed tap; the
//     last lane of a warp reads the next warp's values from shared memory), and the basis-MU
//     weights A = P / lambda^2 and C = (taps counted) / lambda stay in registers.
// Frames at or past J hold y = 0 (and 1/lambda = 0 past J), so every masked term of Eqs. 5,
// 8, 17 and 18 vanishes without a test.
#pragma once

#include "phases.cuh"

namespace ctf {

// The default tap layout of M rows over N sources, at compile time.
template <int M, int N>
struct Taps {
    static_assert(N >= 1 && N <= M, "1 <= N <= M");
    __host__ __device__ static constexpr int Ln(int n) { return M / N + (n < M % N ? 1 : 0); }
    __host__ __device__ static constexpr int row0(int n) { return n * (M / N) + (n < M % N ? n : M % N); }
    __host__ __device__ static constexpr int src(int r)
    {
        int n = 0;
        while (n + 1 < N && r >= row0(n + 1)) ++n;
        return n;
    }
    __host__ __device__ static constexpr int tap(int r) { return r - row0(src(r)); }
    static constexpr int LMAX = M / N + (M % N ? 1 : 0);
};

constexpr int kContigFpt = 8;          // frames per thread
constexpr int kContigMaxThreads = 512; // J <= 4096

// Shared memory of one block (floats): the staged 1/lambda [N][8 + Jp] (8 zero frames in front),
// ISS partials [2][NW][32], basis-MU partials [NW][N][G][8] (G = groups of 4 bases), row-power
// partials [NW][8], the warps' first |y|^2 values [NW][M][4], the bases of the bin [N][B], the
// sweep's normalisers [8].
struct ContigSmem {
    int wst, red, mu, rp, head, tpre, scr, total;
};

__host__ __device__ inline ContigSmem contig_smem_layout(int M, int N, int B, int Jp, int nt)
{
    const int NW = nt / 32, G = contig_groups(B);
    ContigSmem c;
    c.wst = 0;
    c.red = c.wst + N * (kLPad + Jp);
    c.mu = c.red + 2 * NW * 32;
    c.rp = c.mu + NW * N * G * 8;
    c.head = c.rp + NW * 8;
    c.tpre = c.head + NW * M * 4;
    c.scr = c.tpre + N * B;
    c.total = (c.scr + CTFMNMF_MAX_M + 3) & ~3;
    return c;
}

// The 16-float window w_n(j0 - 8 .. j0 + 7) of the staged (and normalisation-scaled) 1/lambda.
__device__ __forceinline__ void load_window(const float* wst_n, int j0, bool active, float (&w)[16])
{
    if (active) {
        const float4* p = reinterpret_cast<const float4*>(wst_n + j0);   // wst_n + kLPad + j0 - 8
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = p[q];
            w[4 * q] = v.x;
            w[4 * q + 1] = v.y;
            w[4 * q + 2] = v.z;
            w[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] = 0.f;
    }
}

// One bin (Sec. III) by the whole block: rows and W_i with the pending normalisation applied,
// the ISS sweep (Eqs. 11-16) with its FP64 normalisers, rows, W_i, P and T stored, per-bin row
// powers in FP64, the |det W_i| factor folded into the running log-det product.
template <int M, int N, int GB>
__device__ __forceinline__ void contig_bin_body(const Shape& s, const State& d, const int i, float* smem,
                                                const int v_tap0)
{
    using TP = Taps<M, N>;
    constexpr int FPT = kContigFpt;
    constexpr int NV = 3 * M - 2;                 // d_p (M real) + n_p, p != r (M - 1 complex)
    constexpr int VP = pow2_at_least(NV);
    constexpr int LM = TP::LMAX;
    static_assert(LM <= 4, "at most 4 taps per source here");
    static_assert(GB == 1 || GB == 3 || GB == 4 || GB == 8, "bases groups: 1, 3, 4 or 8");
    const int J = s.J, Jp = s.Jp, B = s.B;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = nt >> 5;
    const Grp g{tid, nt, 0};
    const ContigSmem L = contig_smem_layout(M, N, B, Jp, nt);
    float* wst = smem + L.wst;
    float* red = smem + L.red;
    float* mus = smem + L.mu;
    float* rps = smem + L.rp;
    float* head = smem + L.head;
    float* tpre = smem + L.tpre;
    float* s_scr = smem + L.scr;
    const int LR = kLPad + Jp;
    const int j0 = tid * FPT;
    const bool active = j0 < Jp;                  // Jp is a multiple of 8: all 8 frames or none

    // pending normalisation of the previous iteration (Eqs. 19-21): rows, W, T and 1/lambda
    float sc[M];
#pragma unroll
    for (int r = 0; r < M; ++r) sc[r] = __ldcg(d.scale + r);

    // ---- the bin's rows (16-byte loads) and column tid < M of W_i
    float2 y[M][FPT];
    float2* Yb = d.Y + (size_t)i * M * Jp;
    float2* Wb = d.W + (size_t)i * M * M;
#pragma unroll
    for (int r = 0; r < M; ++r) {
        const float4* src = reinterpret_cast<const float4*>(Yb + (size_t)r * Jp + j0);
#pragma unroll
        for (int q = 0; q < FPT / 2; ++q) {
            // L1-allocating loads: a warp's q-th load uses half of each 32-byte sector it touches,
            // the (q^1)-th the other half, which then comes from L1 instead of L2
            const float4 v = active ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            y[r][2 * q] = make_float2(v.x, v.y);
            y[r][2 * q + 1] = make_float2(v.z, v.w);
        }
    }
    float2 wcol[M];
    if (tid < M) {
#pragma unroll
        for (int p = 0; p < M; ++p) {
            const float2 w = __ldcg(Wb + p * M + tid);
            wcol[p] = make_float2(w.x * sc[p], w.y * sc[p]);
        }
    }
    // ---- the bin's bases (used at the end)
    for (int t = tid; t < N * B; t += nt) {
        const int n = t / B, k = t - n * B;
        tpre[t] = __ldcg(d.T + (size_t)n * s.FBp + (size_t)i * B + k);
    }
    // ---- stage 1/lambda (cp.async, zero front pad), then scale the entries this thread copied by
    //      mu_{(n,0)}^2 (the stored 1/lambda is formed from the bases before the normalisation)
    {
        const float4* src = reinterpret_cast<const float4*>(d.invlam + (size_t)i * N * Jp);
        float4* dst = reinterpret_cast<float4*>(wst);
        const int LR4 = LR >> 2, J4 = Jp >> 2, P4 = kLPad >> 2;
#pragma unroll
        for (int n = 0; n < N; ++n)
            for (int o = tid; o < LR4; o += nt) {
                if (o < P4) dst[n * LR4 + o] = make_float4(0.f, 0.f, 0.f, 0.f);
                else cp_async16(dst + n * LR4 + o, src + (size_t)n * J4 + o - P4);
            }
        cp_async_wait();
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const float s0 = sc[TP::row0(n)];
            const float fac = 1.0f / (s0 * s0);
            for (int o = tid; o < LR4; o += nt) {
                if (o < P4) continue;
                float4 v = dst[n * LR4 + o];
                v = make_float4(scaled_invlam(v.x, fac), scaled_invlam(v.y, fac), scaled_invlam(v.z, fac),
                                scaled_invlam(v.w, fac));
                dst[n * LR4 + o] = v;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
        for (int f = 0; f < FPT; ++f) y[r][f] = make_float2(y[r][f].x * sc[r], y[r][f].y * sc[r]);
    grp_sync(g);

    // ---- ISS sweep (Eqs. 11-16): step r takes d_p = sum phi_p |y_r|^2 and n_p = sum phi_p y_p y_r^*
    //      over the bin's frames (z_p = n_p / d_p, p != r; the normaliser of row r, formed in FP64
    //      after the sweep, is applied then: every later step is homogeneous in row r)
    float detf = 1.0f;
#pragma unroll
    for (int r = 0; r < M; ++r) {
        float a[VP];
#pragma unroll
        for (int k = 0; k < VP; ++k) a[k] = 0.f;
        float pr[FPT];
#pragma unroll
        for (int f = 0; f < FPT; ++f) pr[f] = abs2(y[r][f]);
#pragma unroll
        for (int n = 0; n < N; ++n) {
            float w[16];                              // w[8 + k] = 1/lambda_n(j0 + k)
            load_window(wst + n * LR, j0, active, w);
#pragma unroll
            for (int l = 0; l < TP::Ln(n); ++l) {
                const int p = TP::row0(n) + l;
#pragma unroll
                for (int f = 0; f < FPT; ++f) {
                    const float ph = w[8 + f - l];    // phi_p(j0 + f), zero where j0 + f < l
                    a[p] = fmaf(ph, pr[f], a[p]);
                    if (p != r) {
                        const int c = M + 2 * (p - (p > r ? 1 : 0));
                        const float2 cc = cmul_conj(y[p][f], y[r][f]);
                        a[c] = fmaf(ph, cc.x, a[c]);
                        a[c + 1] = fmaf(ph, cc.y, a[c + 1]);
                    }
                }
            }
        }
        reduce_scatter<VP>(a, lane);
        float* rb = red + (r & 1) * NW * 32;
        if ((lane & (32 / VP - 1)) == 0) rb[warp * 32 + lane / (32 / VP)] = a[0];
        grp_sync(g);
        float tk = 0.f;
        for (int w = 0; w < NW; ++w) tk += rb[w * 32 + (lane & (VP - 1))];
        float tot[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = __shfl_sync(0xffffffffu, tk, k);
        if (tid == 0) s_scr[r] = tot[r];               // J q_r, inverted after the sweep
        float2 z[M];
#pragma unroll
        for (int p = 0; p < M; ++p) {
            z[p] = make_float2(0.f, 0.f);
            if (p != r && tot[p] > 0.f) {
                const int c = M + 2 * (p - (p > r ? 1 : 0));
                const float inv = 1.0f / tot[p];
                z[p] = make_float2(tot[c] * inv, tot[c + 1] * inv);
            }
        }
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const float2 yr = y[r][f];
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                y[p][f].x -= z[p].x * yr.x - z[p].y * yr.y;
                y[p][f].y -= z[p].x * yr.y + z[p].y * yr.x;
            }
        }
        if (tid < M) {
            const float2 wr = wcol[r];
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                wcol[p].x -= z[p].x * wr.x - z[p].y * wr.y;
                wcol[p].y -= z[p].x * wr.y + z[p].y * wr.x;
            }
        }
    }
    // the first LM - 1 |y|^2 of each warp's lane 0 (before the normalisers), for the delayed
    // power of the previous warp's last lane
    if (lane == 0) {
#pragma unroll
        for (int p = 0; p < M; ++p)
#pragma unroll
            for (int k = 0; k < LM - 1; ++k) head[(warp * M + p) * 4 + k] = abs2(y[p][k]);
    }
    // the FP64 normalisers of all rows by warp 0, one row per lane (an FP64 instruction costs the
    // same for one lane as for 32 on this GPU), published with one barrier
    if (warp == 0) {
        __syncwarp();
        const float scv = iss_normaliser(lane < M ? s_scr[lane] : 0.f, s.invJ);
        __syncwarp();
        if (lane < M) s_scr[lane] = scv;
    }
    grp_sync(g);
    float scr[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
        scr[r] = s_scr[r];
        detf *= scr[r];
#pragma unroll
        for (int f = 0; f < FPT; ++f) y[r][f] = make_float2(y[r][f].x * scr[r], y[r][f].y * scr[r]);
        if (tid < M) wcol[r] = make_float2(wcol[r].x * scr[r], wcol[r].y * scr[r]);
    }

    // ---- store the rows (16-byte stores) and W_i; |y|^2 and the row-power partials
    if (active) {
#pragma unroll
        for (int r = 0; r < M; ++r) {
            float4* dst = reinterpret_cast<float4*>(Yb + (size_t)r * Jp + j0);
#pragma unroll
            for (int q = 0; q < FPT / 2; ++q)
                __stcg(dst + q, make_float4(y[r][2 * q].x, y[r][2 * q].y, y[r][2 * q + 1].x, y[r][2 * q + 1].y));
        }
    }
    if (tid < M) {
#pragma unroll
        for (int p = 0; p < M; ++p) __stcg(Wb + p * M + tid, wcol[p]);
    }
    float sq[M][FPT];
    constexpr int VR = pow2_at_least(M);
    float rp[VR];
#pragma unroll
    for (int r = 0; r < VR; ++r) rp[r] = 0.f;
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            sq[r][f] = abs2(y[r][f]);
            rp[r] += sq[r][f];
        }

    // ---- per source: delayed power P_n(j) = sum_{l < L_n, j + l < J} |y_{(n,l)}(j + l)|^2,
    //      basis-MU weights A = P / lambda^2 and C = (taps counted) / lambda (Eq. 17), P stored
    //      for the activation update (|y_{(n,0)}|^2 for the tap-0 form), then the sums of Eq. 17
    //      over the thread's frames in groups of 4 bases, reduced over the warp
#pragma unroll
    for (int n = 0; n < N; ++n) {
        const int r0 = TP::row0(n);
        float P[FPT];
#pragma unroll
        for (int f = 0; f < FPT; ++f) P[f] = sq[r0][f];
#pragma unroll
        for (int l = 1; l < TP::Ln(n); ++l) {
            const int p = r0 + l;
#pragma unroll
            for (int f = 0; f + l < FPT; ++f) P[f] += sq[p][f + l];
#pragma unroll
            for (int k = 0; k < l; ++k) {             // the next thread's frame j0 + 8 + k
                float v = __shfl_down_sync(0xffffffffu, sq[p][k], 1);
                if (lane == 31) v = warp + 1 < NW ? head[((warp + 1) * M + p) * 4 + k] * (scr[p] * scr[p]) : 0.f;
                P[FPT - l + k] += v;
            }
        }
        float w[16];
        load_window(wst + n * LR, j0, active, w);
        float A[FPT], C[FPT];
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = j0 + f;
            const float cnt = j < J ? (float)min(TP::Ln(n), J - j) : 0.f;
            const float wf = w[8 + f];
            A[f] = P[f] * wf * wf;
            C[f] = cnt * wf;
        }
        if (active) {
            float4* Pp = reinterpret_cast<float4*>(d.P + ((size_t)i * N + n) * Jp + j0);
            float pv[FPT];
#pragma unroll
            for (int f = 0; f < FPT; ++f) pv[f] = v_tap0 ? sq[r0][f] : P[f];
            __stcg(Pp, make_float4(pv[0], pv[1], pv[2], pv[3]));
            __stcg(Pp + 1, make_float4(pv[4], pv[5], pv[6], pv[7]));
        }
        // the sums of every base of the source: GB groups of 4 (compile time, so that all the
        // source's V loads are independent and in flight together), one reduce-scatter
        const float* Vn = d.V + (size_t)n * B * Jp + j0;
        constexpr int NA = 8 * GB;                    // [group][num 4 | den 4]
        constexpr int VA = pow2_at_least(NA);
        float acc[VA];
#pragma unroll
        for (int q = 0; q < VA; ++q) acc[q] = 0.f;
#pragma unroll
        for (int k = 0; k < 4 * GB; ++k) {
            if (k < B && active) {
                const float4* vp = reinterpret_cast<const float4*>(Vn + (size_t)k * Jp);
                const float4 v0 = __ldg(vp), v1 = __ldg(vp + 1);
                const int a = 8 * (k >> 2) + (k & 3);
                acc[a] = fmaf(v0.x, A[0], fmaf(v0.y, A[1], fmaf(v0.z, A[2], fmaf(v0.w, A[3],
                         fmaf(v1.x, A[4], fmaf(v1.y, A[5], fmaf(v1.z, A[6], v1.w * A[7])))))));
                acc[a + 4] = fmaf(v0.x, C[0], fmaf(v0.y, C[1], fmaf(v0.z, C[2], fmaf(v0.w, C[3],
                             fmaf(v1.x, C[4], fmaf(v1.y, C[5], fmaf(v1.z, C[6], v1.w * C[7])))))));
            }
        }
        if constexpr (VA <= 32) {
            reduce_scatter<VA>(acc, lane);
            if ((lane & (32 / VA - 1)) == 0) {
                const int v = lane / (32 / VA);
                if (v < NA) mus[(warp * N + n) * NA + v] = acc[0];
            }
        } else {                                      // 8 groups (B > 16): two halves of 32
            float lo[32], hi[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                lo[q] = acc[q];
                hi[q] = acc[32 + q];
            }
            reduce_scatter<32>(lo, lane);
            reduce_scatter<32>(hi, lane);
            mus[(warp * N + n) * NA + lane] = lo[0];
            mus[(warp * N + n) * NA + 32 + lane] = hi[0];
        }
    }
    reduce_scatter<VR>(rp, lane);
    if ((lane & (32 / VR - 1)) == 0) rps[warp * 8 + lane / (32 / VR)] = rp[0];
    grp_sync(g);

    // ---- basis MU (Eq. 17) with the pending scale of the bases, the row powers in FP64 (Eq. 19),
    //      the |det W_i| factor (Eq. 13) of the sweep and of the pending scale
    for (int t = tid; t < N * B; t += nt) {
        const int n = t / B, k = t - n * B;
        const int slot = n * 8 * GB + 8 * (k >> 2) + (k & 3);
        float num = 0.f, den = 0.f;
        for (int w = 0; w < NW; ++w) {
            num += mus[w * N * 8 * GB + slot];
            den += mus[w * N * 8 * GB + slot + 4];
        }
        float s0 = sc[0];
#pragma unroll
        for (int nn = 1; nn < N; ++nn)
            if (n == nn) s0 = sc[TP::row0(nn)];
        const float tcur = tpre[t] * (s0 * s0);
        const float tn = (den > 0.f) ? tcur * sqrtf(num / den) : tcur;
        __stcg(d.T + (size_t)n * s.FBp + (size_t)i * B + k, fmaxf(tn, s.floor_nmf));
    }
    if (tid < M) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += (double)rps[w * 8 + tid];
        __stcg(d.mupart + (size_t)i * M + tid, t);
    }
    if (tid == 0) d.detb[i] = det_factor<M>(detf, sc);   // folded by the frame phase
}

// Two-kernel path: one block per bin.
template <int M, int N, int GB>
__global__ void __launch_bounds__(kContigMaxThreads, 1) contig_bin_kernel(const Shape s, const State d, const int v_tap0)
{
    extern __shared__ float4 csm4[];
#ifdef CTFMNMF_DEBUG
    if ((int)blockIdx.x >= s.F || (int)blockDim.x * kContigFpt < s.Jp) {
        if (threadIdx.x == 0) atomicOr(d.flag + 3, 1);
        return;
    }
#endif
    contig_bin_body<M, N, GB>(s, d, blockIdx.x, reinterpret_cast<float*>(csm4), v_tap0);
}

// Batched form: one block per (mixture, bin) work item, the mixture's shape and buffers from
// the descriptor table.
template <int M, int N, int GB>
__global__ void __launch_bounds__(kContigMaxThreads, 1) batch_contig_bin_kernel(const MixDesc* __restrict__ mixes,
                                                                                const int2* __restrict__ work,
                                                                                const int v_tap0)
{
    extern __shared__ float4 csm4[];
    __shared__ MixDesc md;
    const int2 w = work[blockIdx.x];
    {
        const int* src = reinterpret_cast<const int*>(mixes + w.x);
        int* dst = reinterpret_cast<int*>(&md);
        for (int e = threadIdx.x; e < (int)(sizeof(MixDesc) / sizeof(int)); e += blockDim.x) dst[e] = src[e];
    }
    __syncthreads();
#ifdef CTFMNMF_DEBUG
    if (w.y < 0 || w.y >= md.s.F || (int)blockDim.x * kContigFpt < md.s.Jp) {
        if (threadIdx.x == 0) atomicOr(md.d.flag + 3, 1);
        return;
    }
#endif
    contig_bin_body<M, N, GB>(md.s, md.d, w.y, reinterpret_cast<float*>(csm4), v_tap0);
}

}  // namespace ctf
