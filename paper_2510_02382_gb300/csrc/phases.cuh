// Device code of one CTF-MNMF-ISS iteration, shared by the two-kernel path
// (bin_phase.cu, kernels.cu) and the persistent kernel (persistent.cu).
//
// A "group" is a set of warps of one CTA that works on one bin (bin phase) or one
// (8-frame tile, source) item (frame phase) and synchronises on its own named barrier.
//
// Data written by other CTAs earlier in the same launch (1/lambda, V, T, P, row powers)
// is read with ld.global.cg (L2, never a possibly stale L1 line).
#pragma once

#include "internal.cuh"

namespace ctf {

constexpr int kLPad = 8;        // zero frames in front of each staged 1/lambda row (taps <= 8)
constexpr int kFrameTile = 8;   // frames per frame-phase item

struct Grp {
    int tid;   // thread index inside the group
    int nt;    // threads in the group (multiple of 32)
    int bar;   // named barrier id (0 when the group is the whole CTA)
};

__device__ __forceinline__ void grp_sync(const Grp& g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(g.bar), "r"(g.nt) : "memory");
}

__host__ __device__ constexpr int pow2_at_least(int v) { return v <= 1 ? 1 : 2 * pow2_at_least((v + 1) / 2); }

// Warp reduce-scatter of V values (V a power of two <= 32): on return a[0] of lane l holds
// the warp-wide sum of value index l / (32 / V). log2(V) halving levels exchange half of the
// remaining values each, then a butterfly finishes the single value.
template <int V>
__device__ __forceinline__ void reduce_scatter(float (&a)[V], int lane)
{
#pragma unroll
    for (int lev = 0; (V >> lev) > 1; ++lev) {
        const int o = 16 >> lev, cnt = V >> lev;
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < cnt / 2; ++q) {
            const float send = hi ? a[q] : a[q + cnt / 2];
            const float keep = hi ? a[q + cnt / 2] : a[q];
            a[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 / V; o >= 1; o >>= 1) a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
}

// ---------------------------------------------------------------------------------------
// Bin phase: shared memory of a group (floats), ragged sizes rounded so float4 views align
struct BinSmem {
    int ils, cw, sq, red, red2, tpre, scr, total;   // offsets (floats)
};

__host__ __device__ inline BinSmem bin_smem_layout(int M, int N, int Jp, int nt)
{
    const int NW = nt / 32;
    BinSmem b;
    b.ils = 0;                                   // [N][kLPad + Jp]
    b.cw = b.ils + N * (kLPad + Jp);             // [N][Jp]
    b.sq = b.cw + N * Jp;                        // [M][Jp]
    b.red = b.sq + M * Jp;                       // [2][NW][32]   ISS partials
    b.red2 = b.red + 2 * NW * 32;                // [NW][N][2][32] basis-update partials
    b.tpre = b.red2 + NW * N * 2 * 32;           // [N * B] this bin's bases, prefetched
    b.scr = b.tpre + N * CTFMNMF_MAX_B;          // [8] the sweep's normalisers 1 - z_r
    b.total = b.scr + CTFMNMF_MAX_M;             // (row powers [NW][8] reuse red)
    b.total = (b.total + 3) & ~3;
    return b;
}

// Entry (a, b) of the Hermitian Q_r stored as M real diagonal entries, then (re, im) of
// Q_r[a][b] for a < b in row-major pair order.
template <int M>
__device__ __forceinline__ void q_entry(const float* Qr, int a, int b, double& re, double& im)
{
    if (a == b) {
        re = Qr[a];
        im = 0.0;
        return;
    }
    const int lo = min(a, b), hi = max(a, b);
    const int pq = lo * M - lo * (lo + 1) / 2 + (hi - lo - 1);
    re = Qr[M + 2 * pq];
    im = a < b ? (double)Qr[M + 2 * pq + 1] : -(double)Qr[M + 2 * pq + 1];
}

// The IP sweep of Eqs. 9-10 for one bin, in FP64 by one warp (all 32 lanes call it): for
// r = 0..M-1 in order, solve (W Q_r) x = e_r, scale by s = (x^H Q_r x)^{-1/2}, set row r of
// W to s x^H. Lane p (M + 1) + q holds entry (p, q) of the augmented matrix [W Q_r | e_r]
// (and W[p][q] for q < M); Gauss-Jordan elimination with partial pivoting (the row of
// largest |a|^2 in the column, the first on ties, swapped with the pivot row) leaves x in
// column M. Qs[r][.] holds Q_r (see q_entry); W (M x M floats, row r = w_r^H) is updated in
// place. A singular W Q_r (a bin without energy, or a covariance that FP32 left without
// full rank) or x^H Q_r x <= 0 leaves that row unchanged.
// *ratio_out = |det W_new| / |det W_old|, without a determinant: replacing row r of W by
// s x^H is the rank-one update W + e_r d^H, and by the matrix determinant lemma
// det W_new / det W = 1 + d^H W^{-1} e_r = s x^H Q_r x (W^{-1} e_r = Q_r x), so each applied
// row contributes the real factor (x^H Q_r x)^{1/2}.
template <int M>
__device__ __forceinline__ void ip_solve_warp(const float* Qs, float2* W, float* ratio_out, const int lane)
{
    constexpr int NQ = M * M, C = M + 1;
    static_assert(M * C <= 32, "one lane per entry of the augmented matrix");
    const unsigned full = 0xffffffffu;
    const int p = lane / C, q = lane - p * C;
    const bool wl = p < M && q < M;                 // lanes holding W[p][q]
    auto at = [](int row, int col) { return min(row * C + col, 31); };
    double wre = 0.0, wim = 0.0;
    if (wl) {
        const float2 w = W[p * M + q];
        wre = w.x;
        wim = w.y;
    }
    double ratio = 1.0;
#pragma unroll
    for (int r = 0; r < M; ++r) {
        const float* Qr = Qs + r * NQ;
        // A[p][q] = sum_k W[p][k] Q_r[k][q]; column M is e_r
        double ar = 0.0, ai = 0.0;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const double wkr = __shfl_sync(full, wre, at(p, k)), wki = __shfl_sync(full, wim, at(p, k));
            double qr = 0.0, qi = 0.0;
            if (wl) q_entry<M>(Qr, k, q, qr, qi);
            ar += wkr * qr - wki * qi;
            ai += wkr * qi + wki * qr;
        }
        if (q == M) {
            ar = p == r ? 1.0 : 0.0;
            ai = 0.0;
        }
        bool ok = true;
#pragma unroll
        for (int c = 0; c < M; ++c) {
            const double mag = ar * ar + ai * ai;
            int piv = c;
            double best = __shfl_sync(full, mag, at(c, c));
#pragma unroll
            for (int pp = c + 1; pp < M; ++pp) {
                const double m = __shfl_sync(full, mag, at(pp, c));
                if (m > best) {
                    best = m;
                    piv = pp;
                }
            }
            if (!(best > 0.0)) {                    // the same decision on every lane
                ok = false;
                break;
            }
            const int src = p == c ? piv : (p == piv ? c : p);
            const double sr = __shfl_sync(full, ar, at(src, q)), si = __shfl_sync(full, ai, at(src, q));
            ar = sr;
            ai = si;
            const double pr = __shfl_sync(full, ar, at(c, c)), pim = __shfl_sync(full, ai, at(c, c));
            const double im2 = 1.0 / best;
            const double ir = pr * im2, ii = -pim * im2;          // 1 / pivot
            const double cr = __shfl_sync(full, ar, at(c, q)), ci = __shfl_sync(full, ai, at(c, q));
            const double fr = __shfl_sync(full, ar, at(p, c)), fi = __shfl_sync(full, ai, at(p, c));
            const double nr = cr * ir - ci * ii, ni = cr * ii + ci * ir;   // pivot row, scaled
            if (p == c) {
                ar = nr;
                ai = ni;
            } else {
                ar -= fr * nr - fi * ni;
                ai -= fr * ni + fi * nr;
            }
        }
        if (!ok) continue;
        // x^H Q_r x: lane (a, b) adds conj(x_a) Q_r[a][b] x_b
        const double xbr = __shfl_sync(full, ar, at(q, M)), xbi = __shfl_sync(full, ai, at(q, M));
        const double xar = __shfl_sync(full, ar, at(p, M)), xai = __shfl_sync(full, ai, at(p, M));
        double term = 0.0;
        if (wl) {
            double qr, qi;
            q_entry<M>(Qr, p, q, qr, qi);
            const double ur = qr * xbr - qi * xbi, ui = qr * xbi + qi * xbr;
            term = xar * ur + xai * ui;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) term += __shfl_xor_sync(full, term, o);
        if (!(term > 0.0)) continue;                // the same sum on every lane
        const double sc = rsqrt(term);
        ratio *= term * sc;
        if (wl && p == r) {                         // row r = s x^H
            wre = xbr * sc;
            wim = -xbi * sc;
        }
    }
    if (wl) W[p * M + q] = make_float2((float)wre, (float)wim);
    if (lane == 0) *ratio_out = (float)ratio;
}

// One CTF-MNMF-ISS bin update (Sec. III) for bin i by group g.
//   in:  y  = the bin's rows with the pending normalisation applied (frames g.tid + f*g.nt)
//        wcol (threads g.tid < M) = column g.tid of W_i with the pending scale applied
//        scale[r] = pending 1/mu_r (for T: T'' = T * scale_{(n,0)}^2, and for the stored
//        1/lambda: times scale_{(n,0)}^{-2})
//   out: the swept rows and W_i (Eqs. 11-16) stored to Ydst [M][Jp] / Wdst [M][M] (HBM when
//        GLOBAL, else a shared-memory copy); T[i] by the basis MU (Eq. 17);
//        P[i] (delayed power, or |y_{(n,0)}|^2 for the tap-0 activation update);
//        mupart[i][r] = sum_j |y_r(j)|^2 (FP64);
//        returns prod_r (1 - z_r), the factor of |det W_i| (Eq. 13).
// IP = true replaces the ISS sweep by the IP update of Eqs. 9-10 (M <= 4): the weighted
// covariances Q_r (Eq. 8) of the kept observation d.X, the sequential solves (ip_solve_warp),
// then y = W x; the return value is then |det W_new| / |det W_old|.
// VPRE = true loads the first V column of the basis update ahead of the barrier before it.
template <int M, int FPT, bool GLOBAL, int KB = 16, bool IP = false, bool VPRE = false, bool ONE = false>
__device__ __forceinline__ float bin_body(const Shape& s, const State& d, const int i, const Grp& g,
                                          float* gsm, float2 (&y)[M][FPT], float2 (&wcol)[M],
                                          float2* Ydst, float2* Wdst, const float* scale, const int v_tap0)
{
    constexpr int NV = 3 * M - 2;                 // d_p (M real) + n_p, p != r (M-1 complex)
    constexpr int VP = pow2_at_least(NV);
    const int J = s.J, Jp = s.Jp, N = s.N, B = s.B;
    const int LR = kLPad + Jp;
    const int lane = g.tid & 31, warp = g.tid >> 5, NW = g.nt >> 5;
    const BinSmem L = bin_smem_layout(M, N, Jp, g.nt);
    float* ils = gsm + L.ils;
    float* Cw = gsm + L.cw;
    float* sq = gsm + L.sq;
    float* red = gsm + L.red;
    float* red2 = gsm + L.red2;
    float* tpre = gsm + L.tpre;
    float* s_scr = gsm + L.scr;

    // ---- prefetch this bin's bases (used at the end; the load overlaps the staging)
    for (int t = g.tid; t < N * B; t += g.nt) {
        const int n = t / B, k = t - n * B;
        tpre[t] = __ldcg(d.T + (size_t)n * s.FBp + (size_t)i * B + k);
    }

    // ---- stage 1/lambda of this bin (cp.async, 16 bytes per copy; zero front pad). The stored
    //      1/lambda is formed from the bases before the pending normalisation: each thread
    //      scales the entries it copied by mu_{(n,0)}^2 once its own copies have landed.
    {
        const float4* src = reinterpret_cast<const float4*>(d.invlam + (size_t)i * N * Jp);
        float4* dst = reinterpret_cast<float4*>(ils);
        const int LR4 = LR >> 2, J4 = Jp >> 2, P4 = kLPad >> 2;
        for (int n = 0; n < N; ++n)
            for (int o = g.tid; o < LR4; o += g.nt) {
                const int e = n * LR4 + o;
                if (o < P4) dst[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                else cp_async16(dst + e, src + (size_t)n * J4 + o - P4);
            }
        cp_async_wait();
        for (int n = 0; n < N; ++n) {
            const float s0 = scale[s.row0[n]];
            const float fac = 1.0f / (s0 * s0);
            for (int o = g.tid; o < LR4; o += g.nt) {
                if (o < P4) continue;
                float4 v = dst[n * LR4 + o];
                v = make_float4(scaled_invlam(v.x, fac), scaled_invlam(v.y, fac), scaled_invlam(v.z, fac),
                                scaled_invlam(v.w, fac));
                dst[n * LR4 + o] = v;
            }
        }
    }
    grp_sync(g);

    // delayed weights phi_p(j) = 1/lambda_{n(p),i,j-l(p)} (zero for j < l(p)): kept in
    // registers when they fit beside the rows, else read from shared memory at each use
    constexpr bool kPhiReg = M * FPT <= 24;
    constexpr int PR = kPhiReg ? M : 1, PF = kPhiReg ? FPT : 1;
    float phi[PR][PF];
    if constexpr (kPhiReg) {
#pragma unroll
        for (int p = 0; p < M; ++p) {
            const float* row = ils + s.row_n[p] * LR + kLPad - s.row_l[p];
#pragma unroll
            for (int f = 0; f < FPT; ++f) phi[p % PR][f % PF] = row[min(g.tid + f * g.nt, Jp - 1)];  // y = 0 past Jp
        }
    }

    const float invJ = 1.0f / (float)J;
    float detf = 1.0f;
    if constexpr (IP) {
        // ---- IP update (Eqs. 8-10): Q_r from the observation, sequential solves, y = W x
        static_assert(M <= 4, "the IP update is instantiated for M <= 4");
        constexpr int NQ = M * M;                    // M real diagonals + M(M-1)/2 complex pairs
        constexpr int VQ = pow2_at_least(NQ);
        // [M][NQ] covariances, one slot for the determinant ratio, then W [M][M] (even offset);
        // 2 + M NQ + 2 M M <= 98 floats fit the basis-update partials (>= 128), free here
        float* Qs = red2;
        float2* Wm = reinterpret_cast<float2*>(red2 + ((M * NQ + 2) & ~1));
        const float2* Xb = d.X + (size_t)i * M * Jp;
#pragma unroll
        for (int r = 0; r < M; ++r)
#pragma unroll
            for (int f = 0; f < FPT; ++f) {
                const int j = g.tid + f * g.nt;
                y[r][f] = j < Jp ? __ldcg(Xb + (size_t)r * Jp + j) : make_float2(0.f, 0.f);
            }
        if (g.tid < M) {
#pragma unroll
            for (int p = 0; p < M; ++p) Wm[p * M + g.tid] = wcol[p];
        }
#pragma unroll
        for (int r = 0; r < M; ++r) {
            float a[VQ];
#pragma unroll
            for (int k = 0; k < VQ; ++k) a[k] = 0.f;
#pragma unroll
            for (int f = 0; f < FPT; ++f) {
                const float ph = kPhiReg ? phi[r % PR][f % PF]
                                         : ils[s.row_n[r] * LR + kLPad + min(g.tid + f * g.nt, Jp - 1) - s.row_l[r]];
                int pq = 0;
#pragma unroll
                for (int a0 = 0; a0 < M; ++a0) {
                    a[a0] = fmaf(ph, abs2(y[a0][f]), a[a0]);
#pragma unroll
                    for (int b0 = a0 + 1; b0 < M; ++b0, ++pq) {
                        const float2 c = cmul_conj(y[a0][f], y[b0][f]);
                        a[M + 2 * pq] = fmaf(ph, c.x, a[M + 2 * pq]);
                        a[M + 2 * pq + 1] = fmaf(ph, c.y, a[M + 2 * pq + 1]);
                    }
                }
            }
            reduce_scatter<VQ>(a, lane);
            float* rb = red + (r & 1) * NW * 32;
            if ((lane & (32 / VQ - 1)) == 0) rb[warp * 32 + lane / (32 / VQ)] = a[0];
            grp_sync(g);
            if (g.tid < NQ) {
                float t = 0.f;
                for (int w = 0; w < NW; ++w) t += rb[w * 32 + g.tid];
                Qs[r * NQ + g.tid] = t * invJ;
            }
        }
        grp_sync(g);
        if (g.tid < 32) ip_solve_warp<M>(Qs, Wm, Qs + M * NQ, lane);   // the slot after Q is free
        grp_sync(g);
        detf = Qs[M * NQ];
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            float2 xv[M];
#pragma unroll
            for (int c = 0; c < M; ++c) xv[c] = y[c][f];
#pragma unroll
            for (int r = 0; r < M; ++r) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const float2 w = Wm[r * M + c];
                    acc.x += w.x * xv[c].x - w.y * xv[c].y;
                    acc.y += w.x * xv[c].y + w.y * xv[c].x;
                }
                y[r][f] = acc;
            }
        }
        if (g.tid < M) {
#pragma unroll
            for (int p = 0; p < M; ++p) wcol[p] = Wm[p * M + g.tid];
        }
    } else {
    // ---- ISS sweep
#pragma unroll
    for (int r = 0; r < M; ++r) {
        float a[VP];
#pragma unroll
        for (int k = 0; k < VP; ++k) a[k] = 0.f;
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const float2 yr = y[r][f];
            const float pr = abs2(yr);
#pragma unroll
            for (int p = 0; p < M; ++p) {
                const float ph = kPhiReg ? phi[p % PR][f % PF]
                                         : ils[s.row_n[p] * LR + kLPad + min(g.tid + f * g.nt, Jp - 1) - s.row_l[p]];
                a[p] = fmaf(ph, pr, a[p]);
                if (p != r) {
                    const int c = M + 2 * (p - (p > r ? 1 : 0));
                    const float2 cc = cmul_conj(y[p][f], yr);
                    a[c] = fmaf(ph, cc.x, a[c]);
                    a[c + 1] = fmaf(ph, cc.y, a[c + 1]);
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
        // 1 - z_r = q^{-1/2}, q = (1/J) sum_j phi_r |y_r|^2, is formed in FP64 at the end of the
        // sweep from this frame sum (kept in shared memory until then). Row r (of Y and of W) is scaled only then: every later step is
        // linear and homogeneous in it (its z_r is the ratio of a sum linear in y_r to one
        // without it, and its update subtracts z_r times another row), so the deferred scale
        // gives the same rows.
        if (g.tid == 0) s_scr[r] = tot[r];
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
        if (g.tid < M) {
            const float2 wr = wcol[r];
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                wcol[p].x -= z[p].x * wr.x - z[p].y * wr.y;
                wcol[p].y -= z[p].x * wr.y + z[p].y * wr.x;
            }
        }
    }
    // the FP64 normalisers of all rows by warp 0, one row per lane (an FP64 instruction costs
    // the same for one lane as for 32 on this GPU), published with one barrier
    if (warp == 0) {
        __syncwarp();
        const float sc = iss_normaliser(lane < M ? s_scr[lane] : 0.f, s.invJ);
        __syncwarp();
        if (lane < M) s_scr[lane] = sc;
    }
    grp_sync(g);
#pragma unroll
    for (int r = 0; r < M; ++r) {
        const float sc = s_scr[r];
        detf *= sc;
#pragma unroll
        for (int f = 0; f < FPT; ++f) y[r][f] = make_float2(y[r][f].x * sc, y[r][f].y * sc);
        if (g.tid < M) wcol[r] = make_float2(wcol[r].x * sc, wcol[r].y * sc);
    }
    }   // ISS

    // ---- store the swept rows and W_i, |y|^2 to shared memory, per-row power partials
    float rp[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
        rp[r] = 0.f;
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = g.tid + f * g.nt;
            if (j < Jp) {
                const float p2 = abs2(y[r][f]);
                sq[r * Jp + j] = p2;
                rp[r] += p2;
                if (GLOBAL) __stcg(Ydst + (size_t)r * Jp + j, y[r][f]);
                else Ydst[r * Jp + j] = y[r][f];
            }
        }
    }
    if (g.tid < M) {
#pragma unroll
        for (int p = 0; p < M; ++p) {
            if (GLOBAL) __stcg(Wdst + p * M + g.tid, wcol[p]);
            else Wdst[p * M + g.tid] = wcol[p];
        }
    }
    // VPRE: the first column of the first basis-update pass (source 0, bases 0 .. KB-1) into
    // registers now, so that its load overlaps the delayed-power step instead of following
    // the barrier after it (for 8 frames per thread: the rows' registers are free here)
    constexpr bool kVpre = VPRE && FPT == 8 && KB <= 10;
    const int J4 = Jp >> 2;
    float4 vpre[kVpre ? KB : 1];
    if constexpr (kVpre) {
        const float4* V0 = reinterpret_cast<const float4*>(d.V);
#pragma unroll
        for (int k = 0; k < KB; ++k)
            vpre[k] = (g.tid < J4 && k < B) ? V0[(size_t)k * J4 + g.tid] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    grp_sync(g);

    // ---- delayed power and the basis-update weights at this thread's frames; the
    //      P/lambda^2 weight overwrites this thread's own 1/lambda entry in place
    float* Pout = d.P + (size_t)i * N * Jp;
#pragma unroll
    for (int p = 0; p < M; ++p) {
        if (s.row_l[p] != 0) continue;          // tap-0 rows enumerate the sources
        const int n = s.row_n[p];
        const int Lp = s.Ln[n];
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = g.tid + f * g.nt;
            if (j >= Jp) continue;
            float P = 0.f, cnt = 0.f;
#pragma unroll
            for (int l = 0; l < M - p; ++l) {       // a source's taps are rows p .. p+L_n-1
                if (l < Lp && j + l < J) {
                    P += sq[(p + l) * Jp + j + l];
                    cnt += 1.f;
                }
            }
            float* wp = ils + n * LR + kLPad + j;
            const float w = *wp;                // 1/lambda_{n,i,j} (zero past J)
            *wp = P * w * w;
            Cw[n * Jp + j] = cnt * w;
            __stcg(Pout + (size_t)n * Jp + j, v_tap0 ? sq[p * Jp + j] : P);
        }
    }
    grp_sync(g);

    // ---- basis MU (Eq. 17): every thread accumulates num/den of all k over its 4-frame
    //      columns (float4 loads of V through the L1, which the groups of a CTA share; the
    //      grid barrier's acquire orders them after the previous frame phase), then a
    //      reduce-scatter per 16 bases
    for (int n = 0; n < N; ++n) {
        const float4* A4 = reinterpret_cast<const float4*>(ils + n * LR + kLPad);
        const float4* C4 = reinterpret_cast<const float4*>(Cw + n * Jp);
        for (int kb = 0; kb < B; kb += KB) {
            float a[32];                  // a[k] = numerator, a[16 + k] = denominator of base kb + k
#pragma unroll
            for (int k = 0; k < 32; ++k) a[k] = 0.f;
            const float4* Vn = reinterpret_cast<const float4*>(d.V + ((size_t)n * B + kb) * Jp);
            int q = g.tid;
            if constexpr (kVpre) {
                if (n == 0 && kb == 0) {          // this thread's first column: the prefetched V
                    if (q < J4) {
                        const float4 A = A4[q], C = C4[q];
#pragma unroll
                        for (int k = 0; k < KB; ++k) {
                            if (k < B) {
                                const float4 v = vpre[k];
                                a[k] = fmaf(v.x, A.x, fmaf(v.y, A.y, fmaf(v.z, A.z, fmaf(v.w, A.w, a[k]))));
                                a[16 + k] = fmaf(v.x, C.x, fmaf(v.y, C.y, fmaf(v.z, C.z, fmaf(v.w, C.w, a[16 + k]))));
                            }
                        }
                    }
                    q += g.nt;
                }
            }
            for (; q < J4; q += g.nt) {
                const float4 A = A4[q], C = C4[q];
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    if (kb + k < B) {
                        const float4 v = Vn[(size_t)k * J4 + q];
                        a[k] = fmaf(v.x, A.x, fmaf(v.y, A.y, fmaf(v.z, A.z, fmaf(v.w, A.w, a[k]))));
                        a[16 + k] = fmaf(v.x, C.x, fmaf(v.y, C.y, fmaf(v.z, C.z, fmaf(v.w, C.w, a[16 + k]))));
                    }
                }
            }
            reduce_scatter<32>(a, lane);
            red2[((warp * N + n) * 2 + kb / KB) * 32 + lane] = a[0];
        }
    }
    // row powers for mu: plain warp sums of M values
#pragma unroll
    for (int r = 0; r < M; ++r) {
        const float v = warp_sum(rp[r]);
        if (lane == 0) red[warp * 8 + r] = v;          // ISS partial buffers are free now
    }
    grp_sync(g);
    for (int t = g.tid; t < N * B; t += g.nt) {
        const int n = t / B, k = t - n * B;
        const int slot = (n * 2 + k / KB) * 32 + (k % KB);
        float num = 0.f, den = 0.f;
        for (int w = 0; w < NW; ++w) {
            num += red2[w * N * 2 * 32 + slot];
            den += red2[w * N * 2 * 32 + slot + 16];
        }
        const float s0 = scale[s.row0[n]];
        float* Tp = d.T + (size_t)n * s.FBp + (size_t)i * B + k;
        const float tcur = tpre[t] * (s0 * s0);
        const float tn = (den > 0.f) ? tcur * sqrtf(num / den) : tcur;
        __stcg(Tp, fmaxf(tn, s.floor_nmf));
    }
    // the bin's row power in FP64 (Eq. 19), by warp 1 where there is one, beside warp 0's
    // basis update above
    const int mt = g.tid - (NW > 1 ? 32 : 0);
    if (mt >= 0 && mt < M) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += (double)red[w * 8 + mt];
        __stcg(d.mupart + (size_t)i * M + mt, t);
    }
    if constexpr (!ONE) grp_sync(g);     // shared memory is reused by the next item of this group
    return detf;
}

// Log-det bookkeeping: |det W_i| is multiplied by `factor` (a product of per-row scales);
// the running product is kept as mantissa ldm[i] in [0.5, 1) and exponent lde[i] so that
// no logarithm is taken inside the iteration; fold_logdet() adds log(ldm) + lde log 2.
__device__ __forceinline__ void logdet_mul(const State& d, int i, double factor)
{
    int e = 0;
    const double m = frexp(__ldcg(d.ldm + i) * factor, &e);
    d.ldm[i] = m;
    d.lde[i] = __ldcg(d.lde + i) + e;
}

// Load bin i's rows (frames g.tid + f*g.nt; zero past Jp) and column g.tid < M of W_i,
// multiplied by the pending scale. GLOBAL: from HBM/L2 (ld.global.cg), else from a
// shared-memory copy with the same [M][Jp] / [M][M] layout.
template <int M, int FPT, bool GLOBAL>
__device__ __forceinline__ void load_bin(const int Jp, const float2* Ysrc, const float2* Wsrc, const Grp& g,
                                         const float* scale, float2 (&y)[M][FPT], float2 (&wcol)[M])
{
#pragma unroll
    for (int r = 0; r < M; ++r) {
        const float sc = scale[r];
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = g.tid + f * g.nt;
            float2 v = make_float2(0.f, 0.f);
            if (j < Jp) v = GLOBAL ? __ldcg(Ysrc + (size_t)r * Jp + j) : Ysrc[r * Jp + j];
            y[r][f] = make_float2(v.x * sc, v.y * sc);
        }
    }
    if (g.tid < M) {
#pragma unroll
        for (int p = 0; p < M; ++p) {
            const float2 w = GLOBAL ? __ldcg(Wsrc + p * M + g.tid) : Wsrc[p * M + g.tid];
            wcol[p] = make_float2(w.x * scale[p], w.y * scale[p]);
        }
    }
}

// load_bin in two halves, so that the row loads need not wait for the pending scale: the
// unscaled rows (frames g.tid + f*g.nt; zero past Jp) and column g.tid < M of W_i from
// HBM/L2 first, then, once the scale is in shared memory, the multiplication.
template <int M, int FPT>
__device__ __forceinline__ void load_bin_unscaled(const int Jp, const float2* Ysrc, const float2* Wsrc, const Grp& g,
                                                  float2 (&y)[M][FPT], float2 (&wcol)[M])
{
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = g.tid + f * g.nt;
            y[r][f] = j < Jp ? __ldcg(Ysrc + (size_t)r * Jp + j) : make_float2(0.f, 0.f);
        }
    if (g.tid < M) {
#pragma unroll
        for (int p = 0; p < M; ++p) wcol[p] = __ldcg(Wsrc + p * M + g.tid);
    }
}

template <int M, int FPT>
__device__ __forceinline__ void apply_bin_scale(const Grp& g, const float* scale, float2 (&y)[M][FPT],
                                                float2 (&wcol)[M])
{
#pragma unroll
    for (int r = 0; r < M; ++r) {
        const float sc = scale[r];
#pragma unroll
        for (int f = 0; f < FPT; ++f) y[r][f] = make_float2(y[r][f].x * sc, y[r][f].y * sc);
    }
    if (g.tid < M) {
#pragma unroll
        for (int p = 0; p < M; ++p) wcol[p] = make_float2(wcol[p].x * scale[p], wcol[p].y * scale[p]);
    }
}

// ---------------------------------------------------------------------------------------
// Frame phase: one (8-frame tile, source n) item by a group. Shared memory (floats):
// Ts [FC][B], Ps [FC][8], red [NW][2*BB][8], vnew [BB][8].
template <int BB>
__host__ __device__ inline int frame_smem_fixed(int nt) { return (nt / 32) * 2 * BB * kFrameTile + BB * kFrameTile; }

// Blocks per SM the batched frame kernel's register budget is sized for (256 threads):
// three up to 10 bases (80 registers, a few spilled; the 48 KB staging area also allows
// three), else the compiler's choice (the 16- and 32-wide accumulators would spill under a
// cap). The single-mixture frame kernel keeps the compiler's choice: its (tile, source)
// items rarely fill two blocks per SM, so the spills would cost without a gain.
template <int BB>
constexpr int frame_min_blocks() { return BB <= 10 ? 3 : 1; }

__host__ __device__ inline int frame_chunk(int avail_floats, int B, int fixed)
{
    return ((avail_floats - fixed) / (B + kFrameTile)) & ~3;   // multiple of 4: Ps stays 16-byte aligned
}

// mu_r^2 = (1/(F J)) sum_i mupart[i][r] (Eq. 19) summed over the bins in FP64, and the pending
// scale 1/mu_r (1 without normalisation, or for a row without energy), by one whole block;
// thread r < M stores it to d.scale[r]. Run once per iteration and mixture, by a block of
// its own, so that its FP64 work (slow on this GPU) is off every other block's path.
// red_cta: shared scratch of (blockDim.x / 32) * CTFMNMF_MAX_M doubles.
// The |det W_i| factor of one bin phase: the ISS normalisers' product detf times the pending
// scale that phase applied to the rows, an FP32 product (detf is one already); the frame
// phase folds it into the FP64 log-det pair (fold_logdet), so no bin block ends on FP64 work.
template <int M>
__device__ __forceinline__ float det_factor(float detf, const float* sc)
{
#pragma unroll
    for (int r = 0; r < M; ++r) detf *= sc[r];
    return detf;
}

// Bins i = first, first + stride, ... of this iteration's factors into the log-det pair.
__device__ __forceinline__ void fold_logdet(const Shape& s, const State& d, int first, int stride)
{
    for (int i = first; i < s.F; i += stride) logdet_mul(d, i, (double)__ldcg(d.detb + i));
}

// FOLD: this block also folds every bin's factor (one block per mixture: the batched form).
template <bool FOLD>
__device__ __forceinline__ void scales_fp64(const Shape& s, const State& d, int normalize, double* red_cta)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int M = s.M, F = s.F;
    double acc[CTFMNMF_MAX_M];
#pragma unroll
    for (int r = 0; r < CTFMNMF_MAX_M; ++r) acc[r] = 0.0;
    for (int i = tid; i < F; i += blockDim.x) {
#pragma unroll
        for (int r = 0; r < CTFMNMF_MAX_M; ++r)
            if (r < M) acc[r] += __ldcg(d.mupart + (size_t)i * M + r);
    }
#pragma unroll
    for (int r = 0; r < CTFMNMF_MAX_M; ++r) {
        if (r >= M) break;
        const double v = warp_sum_d(acc[r]);
        if (lane == 0) red_cta[warp * CTFMNMF_MAX_M + r] = v;
    }
    __syncthreads();
    if (tid < M) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red_cta[w * CTFMNMF_MAX_M + tid];
        const double ms = t / ((double)F * (double)s.J);
        d.scale[tid] = (normalize && ms > 0.0) ? (float)rsqrt(ms) : 1.0f;
    }
    if constexpr (FOLD) fold_logdet(s, d, tid, blockDim.x);
}

// Copy `count` contiguous floats of bases (16-byte aligned source; count rounded up to a
// multiple of 4 stays inside the source block and the staging area) into shared memory.
__device__ __forceinline__ void stage_bases(const float* src, float* dst, int count, const Grp& g)
{
    const int n4 = (count + 3) >> 2;
    for (int e = g.tid; e < n4; e += g.nt)
        cp_async16(reinterpret_cast<float4*>(dst) + e, reinterpret_cast<const float4*>(src) + e);
}

// One frame-phase item (Eq. 18, all-taps form by default, then the next PSD):
//   lambda'_{n,i,j} = sum_k T'[i][n][k] V[n][k][j],  T' = the bases of this iteration,
//   num[k] = sum_i T'[i][n][k] P[i][n][j]/lambda'^2,  den[k] = sum_i T'[i][n][k] c_n(j)/lambda',
//   V[n][k][j] <- max(V sqrt(num/den), floor),
//   1/lambda for the next iteration with T' and the new V; the normalisation of Eqs. 19-21
//   (T'' = T' scale_{(n,0)}^2) is applied to it by the next bin phase.
// Threads: tx = tid & 7 frame of the tile, ty = tid >> 3 bin slice (one frame per thread:
// the variant for many bases, BB = 32).
template <int BB, bool EXACT = false, bool ONE = false>
__device__ __forceinline__ void frame_item_wide(const Shape& s, const State& d, const int item, const Grp& g,
                                           float* gsm, const int FC, const int v_tap0)
{
    const int M = s.M, N = s.N, F = s.F, J = s.J, Jp = s.Jp;
    const int B = EXACT ? BB : s.B;     // EXACT: the bases count is the class width
    (void)M;
    const int ntiles = Jp / kFrameTile;
    const int n = item / ntiles, tile = item - n * ntiles;
    const int j0 = tile * kFrameTile;
    const int tx = g.tid & 7, ty = g.tid >> 3, NY = g.nt >> 3;
    const int lane = g.tid & 31, warp = g.tid >> 5, NW = g.nt >> 5;
    const int j = j0 + tx;
    float* Ts = gsm;                        // [FC][B]
    float* Ps = gsm + FC * B;               // [FC][8]
    float* red = Ps + FC * kFrameTile;      // [NW][2*BB][8]
    float* vnew = red + NW * 2 * BB * kFrameTile;   // [BB][8]

    const bool valid = j < J;
    float vk[BB];
#pragma unroll
    for (int k = 0; k < BB; ++k) vk[k] = (k < B && valid) ? __ldcg(d.V + ((size_t)n * B + k) * Jp + j) : 0.f;
    const float cnt = valid ? (v_tap0 ? 1.f : (float)min(s.Ln[n], J - j)) : 0.f;

    float an[BB], ad[BB];
#pragma unroll
    for (int k = 0; k < BB; ++k) { an[k] = 0.f; ad[k] = 0.f; }
    const float* Tn = d.T + (size_t)n * s.FBp;
    for (int c0 = 0; c0 < F; c0 += FC) {
        const int nb = min(FC, F - c0);
        stage_bases(Tn + (size_t)c0 * B, Ts, nb * B, g);
        for (int e = g.tid; e < nb * 2; e += g.nt) {
            const int ii = e >> 1, h = e & 1;
            cp_async16(reinterpret_cast<float4*>(Ps) + e,
                       reinterpret_cast<const float4*>(d.P + ((size_t)(c0 + ii) * N + n) * Jp + j0) + h);
        }
        cp_async_wait();
        grp_sync(g);
        if (valid) {
            for (int ii = ty; ii < nb; ii += NY) {
                const float* Ti = Ts + ii * B;
                float l0 = 0.f, l1 = 0.f;     // two partial sums: half the dependent chain
#pragma unroll
                for (int k = 0; k < BB; k += 2) {
                    if (k < B) l0 = fmaf(Ti[k], vk[k], l0);
                    if (k + 1 < BB && k + 1 < B) l1 = fmaf(Ti[k + 1], vk[k + 1], l1);
                }
                const float il = recip(fmaxf(l0 + l1, kFloorPsd));
                const float gg = Ps[ii * kFrameTile + tx] * il * il;
                const float hh = cnt * il;
#pragma unroll
                for (int k = 0; k < BB; ++k) {
                    if (k < B) {
                        const float t = Ti[k];
                        an[k] = fmaf(t, gg, an[k]);
                        ad[k] = fmaf(t, hh, ad[k]);
                    }
                }
            }
        }
        grp_sync(g);
    }
    // reduce over the 4 bin slices inside the warp (lanes with equal tx), then over warps
#pragma unroll
    for (int k = 0; k < BB; ++k) {
        if (k >= B) break;
        an[k] += __shfl_xor_sync(0xffffffffu, an[k], 8);
        an[k] += __shfl_xor_sync(0xffffffffu, an[k], 16);
        ad[k] += __shfl_xor_sync(0xffffffffu, ad[k], 8);
        ad[k] += __shfl_xor_sync(0xffffffffu, ad[k], 16);
        if (lane < 8) {
            red[(warp * 2 * BB + k) * kFrameTile + lane] = an[k];
            red[(warp * 2 * BB + BB + k) * kFrameTile + lane] = ad[k];
        }
    }
    grp_sync(g);
    for (int t = g.tid; t < B * kFrameTile; t += g.nt) {
        const int k = t >> 3, x = t & 7;
        const int jj = j0 + x;
        float num = 0.f, den = 0.f;
        for (int w = 0; w < NW; ++w) {
            num += red[(w * 2 * BB + k) * kFrameTile + x];
            den += red[(w * 2 * BB + BB + k) * kFrameTile + x];
        }
        float v = 0.f;
        if (jj < J) {
            float* Vp = d.V + ((size_t)n * B + k) * Jp + jj;
            const float vo = __ldcg(Vp);
            v = (den > 0.f) ? vo * sqrtf(num / den) : vo;
            v = fmaxf(v, s.floor_nmf);
            __stcg(Vp, v);
        }
        vnew[k * kFrameTile + x] = v;
    }
    grp_sync(g);

    // ---- PSD of the next iteration (bases before the normalisation)
#pragma unroll
    for (int k = 0; k < BB; ++k) vk[k] = k < B ? vnew[k * kFrameTile + tx] : 0.f;
    for (int c0 = 0; c0 < F; c0 += FC) {
        const int nb = min(FC, F - c0);
        if (F > FC) {                      // restage the bases chunk (only when chunked)
            stage_bases(Tn + (size_t)c0 * B, Ts, nb * B, g);
            cp_async_wait();
            grp_sync(g);
        }
        for (int ii = ty; ii < nb; ii += NY) {
            const float* Ti = Ts + ii * B;
            float l0 = 0.f, l1 = 0.f;
#pragma unroll
            for (int k = 0; k < BB; k += 2) {
                if (k < B) l0 = fmaf(Ti[k], vk[k], l0);
                if (k + 1 < BB && k + 1 < B) l1 = fmaf(Ti[k + 1], vk[k + 1], l1);
            }
            __stcg(d.invlam + ((size_t)(c0 + ii) * N + n) * Jp + j,
                   valid ? recip(fmaxf(l0 + l1, kFloorPsd)) : 0.f);
        }
        if (F > FC) grp_sync(g);
    }
    if constexpr (!ONE) grp_sync(g);     // shared memory is reused by the next item of this group
}

// The same item with two frames per thread (BB <= 16): each row of bases read from shared
// memory feeds the two frames' PSD and both sums, and the reduction over the 8 bin slices
// of a warp is a three-level reduce-scatter. Threads: tx = tid & 3 owns frames j0 + 2tx
// and j0 + 2tx + 1, ty = tid >> 2 is the bin slice.
template <int BB, bool EXACT = false, bool ONE = false>
__device__ __forceinline__ void frame_item(const Shape& s, const State& d, const int item, const Grp& g,
                                           float* gsm, const int FC, const int v_tap0)
{
    static_assert(BB % 2 == 0 && BB <= 16, "two-frame item needs an even BB <= 16");
    const int N = s.N, F = s.F, J = s.J, Jp = s.Jp;
    const int B = EXACT ? BB : s.B;     // EXACT: the bases count is the class width (no per-k tests)
    const int ntiles = Jp / kFrameTile;
    const int n = item / ntiles, tile = item - n * ntiles;
    const int j0 = tile * kFrameTile;
    const int tx = g.tid & 3, ty = g.tid >> 2, NY = g.nt >> 2;
    const int lane = g.tid & 31, warp = g.tid >> 5, NW = g.nt >> 5;
    const int ja = j0 + 2 * tx;
    float* Ts = gsm;                                // [FC][B]
    float* Ps = gsm + FC * B;                       // [FC][8]
    float* red = Ps + FC * kFrameTile;              // [NW][4 frame pairs][4 BB]
    float* vnew = red + NW * 16 * BB;               // [BB][8]

    const bool va = ja < J, vb = ja + 1 < J;
    float v0[BB], v1[BB];
#pragma unroll
    for (int k = 0; k < BB; ++k) {
        float2 v = make_float2(0.f, 0.f);
        if (k < B) v = __ldcg(reinterpret_cast<const float2*>(d.V + ((size_t)n * B + k) * Jp + ja));
        v0[k] = va ? v.x : 0.f;
        v1[k] = vb ? v.y : 0.f;
    }
    const int Lp = s.Ln[n];
    const float c0 = va ? (v_tap0 ? 1.f : (float)min(Lp, J - ja)) : 0.f;
    const float c1 = vb ? (v_tap0 ? 1.f : (float)min(Lp, J - ja - 1)) : 0.f;

    float acc[4 * BB];        // numerators of frames 0, 1 then denominators of frames 0, 1
#pragma unroll
    for (int k = 0; k < 4 * BB; ++k) acc[k] = 0.f;
    const float* Tn = d.T + (size_t)n * s.FBp;
    for (int cb = 0; cb < F; cb += FC) {
        const int nb = min(FC, F - cb);
        stage_bases(Tn + (size_t)cb * B, Ts, nb * B, g);
        for (int e = g.tid; e < nb * 2; e += g.nt) {
            const int ii = e >> 1, h = e & 1;
            cp_async16(reinterpret_cast<float4*>(Ps) + e,
                       reinterpret_cast<const float4*>(d.P + ((size_t)(cb + ii) * N + n) * Jp + j0) + h);
        }
        cp_async_wait();
        grp_sync(g);
        for (int ii = ty; ii < nb; ii += NY) {
            const float* Ti = Ts + ii * B;
            float t[BB];
#pragma unroll
            for (int k = 0; k < BB; ++k) t[k] = k < B ? Ti[k] : 0.f;
            float l0a = 0.f, l0b = 0.f, l1a = 0.f, l1b = 0.f;
#pragma unroll
            for (int k = 0; k < BB; k += 2) {
                l0a = fmaf(t[k], v0[k], l0a);
                l0b = fmaf(t[k + 1], v0[k + 1], l0b);
                l1a = fmaf(t[k], v1[k], l1a);
                l1b = fmaf(t[k + 1], v1[k + 1], l1b);
            }
            const float i0 = recip(fmaxf(l0a + l0b, kFloorPsd));
            const float i1 = recip(fmaxf(l1a + l1b, kFloorPsd));
            const float2 p = *reinterpret_cast<const float2*>(Ps + ii * kFrameTile + 2 * tx);
            const float g0 = p.x * i0 * i0, g1 = p.y * i1 * i1, h0 = c0 * i0, h1 = c1 * i1;
#pragma unroll
            for (int k = 0; k < BB; ++k) {
                acc[k] = fmaf(t[k], g0, acc[k]);
                acc[BB + k] = fmaf(t[k], g1, acc[BB + k]);
                acc[2 * BB + k] = fmaf(t[k], h0, acc[2 * BB + k]);
                acc[3 * BB + k] = fmaf(t[k], h1, acc[3 * BB + k]);
            }
        }
        grp_sync(g);
    }
    // sum over the 8 bin slices of the warp (lane bits 2..4): three halving levels; lane
    // then holds BB/2 consecutive values starting at `base` for its frame pair tx
#pragma unroll
    for (int lev = 0; lev < 3; ++lev) {
        const int o = 16 >> lev, half = (2 * BB) >> lev;
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < half; ++q) {
            const float send = hi ? acc[q] : acc[q + half];
            const float keep = hi ? acc[q + half] : acc[q];
            acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    {
        const int base = ((lane >> 4) & 1) * 2 * BB + ((lane >> 3) & 1) * BB + ((lane >> 2) & 1) * (BB / 2);
        float* rw = red + (warp * 4 + tx) * 4 * BB + base;
#pragma unroll
        for (int q = 0; q < BB / 2; ++q) rw[q] = acc[q];
    }
    grp_sync(g);
    for (int t = g.tid; t < B * kFrameTile; t += g.nt) {
        const int k = t >> 3, x = t & 7;
        const int jj = j0 + x;
        const int off = (x >> 1) * 4 * BB + (x & 1) * BB + k;
        float num = 0.f, den = 0.f;
        for (int w = 0; w < NW; ++w) {
            num += red[w * 16 * BB + off];
            den += red[w * 16 * BB + off + 2 * BB];
        }
        float v = 0.f;
        if (jj < J) {
            float* Vp = d.V + ((size_t)n * B + k) * Jp + jj;
            const float vo = __ldcg(Vp);
            v = (den > 0.f) ? vo * sqrtf(num / den) : vo;
            v = fmaxf(v, s.floor_nmf);
            __stcg(Vp, v);
        }
        vnew[k * kFrameTile + x] = v;
    }
    grp_sync(g);

    // ---- PSD of the next iteration, bases before the normalisation (two frames per thread)
#pragma unroll
    for (int k = 0; k < BB; ++k) {
        v0[k] = k < B ? vnew[k * kFrameTile + 2 * tx] : 0.f;
        v1[k] = k < B ? vnew[k * kFrameTile + 2 * tx + 1] : 0.f;
    }
    for (int cb = 0; cb < F; cb += FC) {
        const int nb = min(FC, F - cb);
        if (F > FC) {                      // restage the bases chunk (only when chunked)
            stage_bases(Tn + (size_t)cb * B, Ts, nb * B, g);
            cp_async_wait();
            grp_sync(g);
        }
        for (int ii = ty; ii < nb; ii += NY) {
            const float* Ti = Ts + ii * B;
            float l0a = 0.f, l0b = 0.f, l1a = 0.f, l1b = 0.f;
#pragma unroll
            for (int k = 0; k < BB; k += 2) {
                const float ta = k < B ? Ti[k] : 0.f, tb = k + 1 < B ? Ti[k + 1] : 0.f;
                l0a = fmaf(ta, v0[k], l0a);
                l0b = fmaf(tb, v0[k + 1], l0b);
                l1a = fmaf(ta, v1[k], l1a);
                l1b = fmaf(tb, v1[k + 1], l1b);
            }
            const float2 o = make_float2(va ? recip(fmaxf(l0a + l0b, kFloorPsd)) : 0.f,
                                         vb ? recip(fmaxf(l1a + l1b, kFloorPsd)) : 0.f);
            __stcg(reinterpret_cast<float2*>(d.invlam + ((size_t)(cb + ii) * N + n) * Jp + ja), o);
        }
        if (F > FC) grp_sync(g);
    }
    if constexpr (!ONE) grp_sync(g);     // shared memory is reused by the next item of this group
}

}  // namespace ctf
