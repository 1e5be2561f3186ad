// The per-bin adjoint (kernel C of grad.cu) and its launch templates, instantiated once
// per M in grad_bin_m<M>.cu so that the translation units compile in parallel; also the
// small device helpers the backward kernels share.
#pragma once

#include "grad.cuh"
#include "phases.cuh"

namespace ctf {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Sum a[V] over the thread block; every thread finds the sums in out[V] (shared) afterwards.
// red holds (threads / 32) * V floats. The warp stage is a reduce-scatter over the next
// power of two of V values (V - 1 + log2(32 / VP) exchanges instead of 5 V).
template <int V>
__device__ __forceinline__ void block_sum(float (&a)[V], float* red, float* out)
{
    constexpr int VP = pow2_at_least(V);
    static_assert(VP <= 32, "block_sum reduces at most 32 values");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float b[VP];
#pragma unroll
    for (int v = 0; v < VP; ++v) b[v] = v < V ? a[v] : 0.f;
    reduce_scatter<VP>(b, lane);
    constexpr int per = 32 / VP;                  // lanes holding each value's sum
    if ((lane & (per - 1)) == 0 && lane / per < V) red[warp * V + lane / per] = b[0];
    __syncthreads();
    if ((int)threadIdx.x < V) {
        float t = 0.f;
        for (int w = 0; w < nw; ++w) t += red[w * V + threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- C: per-bin adjoint
// Threads per block: up to 256 for FPT <= 2 (three blocks per SM), up to 512 for FPT = 4.
template <int M, int FPT>
__global__ void __launch_bounds__(FPT == 4 ? 512 : 256, FPT == 4 ? 1 : 3)
grad_bin_kernel(const Shape s, const StatePtrs* __restrict__ cur_tab, const StatePtrs* __restrict__ nxt_tab,
                const GradBufs g, const int vstage)
{
    constexpr int VF = 3 * M - 2;   // forward ISS sums per step: d_p, n_p (p != r), q
    constexpr int VB = 2 * M - 1;   // backward ISS sums per step: G_p (p != r), Gs
    constexpr int NB = kGradMaxM * CTFMNMF_MAX_B;
    extern __shared__ float4 gsm4[];
    const int N = s.N, B = s.B, F = s.F, J = s.J, Jp = s.Jp, FBp = s.FBp;
    float* invl = reinterpret_cast<float*>(gsm4);          // [N][Jp] 1/lambda (0 past J)
    float* sq = invl + N * Jp;                             // [M][Jp] |Y1|^2
    float* gS = sq + M * Jp;                               // [N][Jp] dL/d(delayed power)
    float* gl = gS + N * Jp;                               // [N][Jp] dL/dlambda
    float2* y0s = reinterpret_cast<float2*>(gl + N * Jp);  // [M][Jp] rows at the iteration start
    float* Vst = reinterpret_cast<float*>(y0s + M * Jp);   // [N][B][Jp] V, when vstage
    __shared__ float2 Wv[M + 1][M][M];                     // W_i before step r of the sweep
    __shared__ float2 zs[M][M];                            // z of step r
    __shared__ float dsv[M][M];                            // d_p of step r (p != r), q at p = r
    __shared__ float ssv[M];                               // q^{-1/2} of step r
    __shared__ float2 gWs[M][M];                           // running dL/dW_i
    __shared__ float Ti[NB], T1i[NB], gT1[NB], denT[NB], gnTs[NB], gdTs[NB], gTacc[NB];
    __shared__ float red[16 * 16];
    __shared__ float bout[16];
    __shared__ float2 gn_b[M];
    __shared__ float gd_b[M];
    __shared__ float gq_b;
    __shared__ float eas[16 * M];                          // per-warp sums of Re(conj(dL/dY) Y)

    const int i = blockIdx.x, sm = blockIdx.y;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31;
    const StatePtrs cur = cur_tab[sm], nxt = nxt_tab[sm];
    const float* sig = g.sig + sm * M;
    const size_t tb = (size_t)sm * N * FBp;
    const size_t fb = (size_t)sm * N;

    // ---- bases of the bin, dL/dT1 = sigma_0^2 dL/dT' plus the activation MU's part (the
    // per-tile sums of kernel E), the basis-MU denominator, W_i, dL/dW1 = sigma dL/dW'
    const int tiles = (Jp + 31) >> 5;
    for (int t = tid; t < N * B; t += NT) {
        const int n = t / B, k = t - n * B;
        const size_t o = (size_t)n * FBp + (size_t)i * B + k;
        const float s0 = sig[s.row0[n]];
        const float* part = g.actp + ((((size_t)sm * N + n) * tiles) * F + i) * (size_t)(2 * B);
        const size_t tstride = (size_t)F * 2 * B;
        float ga = 0.f, dn = 0.f;
        for (int q = 0; q < tiles; ++q) {
            ga += part[q * tstride + k];
            dn += part[q * tstride + B + k];
        }
        Ti[t] = cur.T[o];
        T1i[t] = nxt.T[o] / (s0 * s0);
        gT1[t] = fmaf(g.gT[tb + o], s0 * s0, ga);
        denT[t] = dn;
        gTacc[t] = 0.f;
    }
    if (tid < M * M) {
        const int p = tid / M, c = tid - p * M;
        Wv[0][p][c] = cur.W[((size_t)i * M + p) * M + c];
        const float2 gw = g.gW[(((size_t)sm * F + i) * M + p) * M + c];
        gWs[p][c] = make_float2(gw.x * sig[p], gw.y * sig[p]);
    }
    // ---- the rows at the start of the iteration; V (when staged); 1/lambda of the iteration's
    // T, V and dL/dS through the activation MU (both from kernel E; [N][F][Jp] planes, so a
    // bin's N rows are Jp apart only within one source)
    {
        const float2* Yc = cur.Y + (size_t)i * M * Jp;
        for (int e = tid; e < M * Jp; e += NT) y0s[e] = Yc[e];
        for (int e = tid; e < N * Jp; e += NT) {
            const int n = e / Jp, j = e - n * Jp;
            const size_t q = ((fb + n) * F + i) * (size_t)Jp + j;
            gS[e] = g.gsa[q];
            invl[e] = g.ilp[q];
        }
        if (vstage)
            for (int e = tid; e < N * B * Jp / 4; e += NT)
                reinterpret_cast<float4*>(Vst)[e] = reinterpret_cast<const float4*>(cur.V)[e];
    }
    __syncthreads();
    const float* Vsrc = vstage ? Vst : cur.V;              // V [N][B][Jp], shared or global
    const float thr = 1.f / kFloorPsd;                     // 1/lambda at (or past) the floor

    auto phi = [&](int p, int j) -> float {   // 1/lambda_{n(p), j - l(p)}, 0 when masked
        const int l = s.row_l[p];
        return (j >= l && j < J) ? invl[s.row_n[p] * Jp + j - l] : 0.f;
    };

    // ---- forward ISS sweep (Eqs. 11-16), keeping z, d, q of every step
    const double invJd = 1.0 / (double)J;
    float2 y[M][FPT];
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = tid + f * NT;
            y[r][f] = j < Jp ? y0s[r * Jp + j] : make_float2(0.f, 0.f);
        }
#pragma unroll
    for (int r = 0; r < M; ++r) {
        float a[VF];
#pragma unroll
        for (int v = 0; v < VF; ++v) a[v] = 0.f;
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = tid + f * NT;
            const float2 yr = y[r][f];
            const float yr2 = abs2(yr);
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                const int q = p < r ? p : p - 1;
                const float ph = phi(p, j);
                const float2 c = cmul_conj(y[p][f], yr);
                a[3 * q] = fmaf(ph, yr2, a[3 * q]);
                a[3 * q + 1] = fmaf(ph, c.x, a[3 * q + 1]);
                a[3 * q + 2] = fmaf(ph, c.y, a[3 * q + 2]);
            }
            a[VF - 1] = fmaf(phi(r, j), yr2, a[VF - 1]);
        }
        block_sum<VF>(a, red, bout);
        if (tid == 0) {
            float2 z[M];
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                const int q = p < r ? p : p - 1;
                const float d = bout[3 * q];
                z[p] = d > 0.f ? make_float2(bout[3 * q + 1] / d, bout[3 * q + 2] / d) : make_float2(0.f, 0.f);
                zs[r][p] = z[p];
                dsv[r][p] = d;
            }
            const float qv = bout[VF - 1] / (float)J;
            const float sr = iss_normaliser(bout[VF - 1], invJd);      // as the forward sweep (FP64)
            z[r] = make_float2(1.f - sr, 0.f);
            zs[r][r] = z[r];
            dsv[r][r] = qv;
            ssv[r] = sr;
#pragma unroll
            for (int c = 0; c < M; ++c) {
                const float2 wr = Wv[r][r][c];
#pragma unroll
                for (int p = 0; p < M; ++p) {
                    const float2 w = Wv[r][p][c];
                    if (p == r) Wv[r + 1][p][c] = make_float2(sr * wr.x, sr * wr.y);
                    else {
                        const float2 zw = cmulf(z[p], wr);
                        Wv[r + 1][p][c] = make_float2(w.x - zw.x, w.y - zw.y);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const float2 yr = y[r][f];
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                const float2 zy = cmulf(zs[r][p], yr);
                y[p][f] = make_float2(y[p][f].x - zy.x, y[p][f].y - zy.y);
            }
            y[r][f] = make_float2(ssv[r] * yr.x, ssv[r] * yr.y);
        }
    }

    // ---- normalisation adjoint: dL/dY1 = sigma (dL/dY' - (e_r / (F J)) Y'), Y' = sigma Y1
    float2 gy[M][FPT];
    {
        const float2* gYb = g.gY + ((size_t)sm * F + i) * M * Jp;
        const double FJ = (double)F * (double)J;
#pragma unroll
        for (int r = 0; r < M; ++r) {
            const float sg = sig[r];
            const float coef = (float)(g.e[sm * M + r] / FJ);
#pragma unroll
            for (int f = 0; f < FPT; ++f) {
                const int j = tid + f * NT;
                float2 v = make_float2(0.f, 0.f);
                if (j < J) {
                    const float2 gp = gYb[(size_t)r * Jp + j];
                    v = make_float2(sg * (gp.x - coef * sg * y[r][f].x), sg * (gp.y - coef * sg * y[r][f].y));
                }
                gy[r][f] = v;
                if (j < Jp) sq[r * Jp + j] = abs2(y[r][f]);
            }
        }
    }
    __syncthreads();

    // delayed power S_n(j) = sum_{l < L_n, j + l < J} |Y1_{(n,l)}(j + l)|^2 and its tap count
    auto delayed = [&](int n, int j, float* S, float* c) {
        float acc = 0.f;
        int cnt = 0;
        const int r0 = s.row0[n], Lq = s.Ln[n];
        for (int l = 0; l < Lq; ++l)
            if (j + l < J) {
                acc += sq[(r0 + l) * Jp + j + l];
                ++cnt;
            }
        *S = acc;
        *c = (float)cnt;
    };

    // ---- basis MU adjoint (Eq. 17): T1 = T R, R = sqrt(numT / denT)
    for (int t = tid; t < N * B; t += NT) {
        const int n = t / B, k = t - n * B;
        const float T = Ti[t], T1 = T1i[t], g1 = gT1[t], dn = denT[t];
        float gTd = 0.f, gn = 0.f, gd = 0.f;
        if (T1 > 1.0001f * s.floor_nmf && T > 0.f && dn > 0.f) {
            const float R = T1 / T, gR = g1 * T;
            gTd = g1 * R;
            gn = gR / (2.f * R * dn);
            gd = -gR * R / (2.f * dn);
        }
        gTacc[t] = gTd;
        gnTs[t] = gn;
        gdTs[t] = gd;
        const size_t o = tb + (size_t)n * FBp + (size_t)i * B + k;
        g.gnT[o] = gn;
        g.gdT[o] = gd;
    }
    __syncthreads();
    for (int n = 0; n < N; ++n) {
        const float* Vn = Vsrc + (size_t)n * B * Jp;
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = tid + f * NT;
            float A = 0.f;
            if (j < J) {
                float S, c;
                delayed(n, j, &S, &c);
                float gA = 0.f, gC = 0.f;
                for (int k = 0; k < B; ++k) {
                    const float vk = Vn[(size_t)k * Jp + j];
                    gA = fmaf(gnTs[n * B + k], vk, gA);
                    gC = fmaf(gdTs[n * B + k], vk, gC);
                }
                const float il = invl[n * Jp + j];
                A = S * il * il;
                const float cc = c * il;
                gS[n * Jp + j] += gA * il * il;
                gl[n * Jp + j] = -2.f * A * il * gA - cc * il * gC;
            } else if (j < Jp) {
                gl[n * Jp + j] = 0.f;
            }
            if (j < Jp) g.aq[((fb + n) * F + i) * (size_t)Jp + j] = A;
        }
    }
    __syncthreads();
    // delayed power -> rows: dL/dY1_{(n,l)}(j) += 2 gS_n(j - l) Y1_{(n,l)}(j)
#pragma unroll
    for (int r = 0; r < M; ++r) {
        const int n = s.row_n[r], l = s.row_l[r];
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = tid + f * NT;
            if (j >= l && j < J) {
                const float w = 2.f * gS[n * Jp + j - l];
                gy[r][f] = make_float2(gy[r][f].x + w * y[r][f].x, gy[r][f].y + w * y[r][f].y);
            }
        }
    }

    // ---- ISS sweep adjoint, steps r = M-1 .. 0
    float gph[M][FPT];
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
        for (int f = 0; f < FPT; ++f) gph[r][f] = 0.f;
#pragma unroll
    for (int r = M - 1; r >= 0; --r) {
        // rows before step r: replay steps 0..r-1 from the iteration start with the stored z
        float2 yw[M][FPT];
#pragma unroll
        for (int p = 0; p < M; ++p)
#pragma unroll
            for (int f = 0; f < FPT; ++f) {
                const int j = tid + f * NT;
                yw[p][f] = j < Jp ? y0s[p * Jp + j] : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int rr = 0; rr < r; ++rr)
#pragma unroll
            for (int f = 0; f < FPT; ++f) {
                const float2 t = yw[rr][f];
#pragma unroll
                for (int p = 0; p < M; ++p) {
                    if (p == rr) continue;
                    const float2 zy = cmulf(zs[rr][p], t);
                    yw[p][f] = make_float2(yw[p][f].x - zy.x, yw[p][f].y - zy.y);
                }
                yw[rr][f] = make_float2(ssv[rr] * t.x, ssv[rr] * t.y);
            }
        float a[VB];
#pragma unroll
        for (int v = 0; v < VB; ++v) a[v] = 0.f;
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const float2 yr = yw[r][f];
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                const int q = p < r ? p : p - 1;
                const float2 c = cmul_conj(gy[p][f], yr);
                a[2 * q] += c.x;
                a[2 * q + 1] += c.y;
            }
            a[VB - 1] = fmaf(gy[r][f].x, yr.x, fmaf(gy[r][f].y, yr.y, a[VB - 1]));
        }
        block_sum<VB>(a, red, bout);
        if (tid == 0) {
            const float sr = ssv[r];
            float gsv = bout[VB - 1];
#pragma unroll
            for (int c = 0; c < M; ++c) gsv = fmaf(gWs[r][c].x, Wv[r][r][c].x, fmaf(gWs[r][c].y, Wv[r][r][c].y, gsv));
            float2 nw[M];
#pragma unroll
            for (int c = 0; c < M; ++c) nw[c] = make_float2(sr * gWs[r][c].x, sr * gWs[r][c].y);
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                const int q = p < r ? p : p - 1;
                float2 gz = make_float2(-bout[2 * q], -bout[2 * q + 1]);
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const float2 t = cmul_conj(gWs[p][c], Wv[r][r][c]);
                    gz = make_float2(gz.x - t.x, gz.y - t.y);
                    const float2 u = cmulf(conjf2(zs[r][p]), gWs[p][c]);
                    nw[c] = make_float2(nw[c].x - u.x, nw[c].y - u.y);
                }
                const float d = dsv[r][p];
                if (d > 0.f) {
                    const float2 z = zs[r][p];
                    gn_b[p] = make_float2(gz.x / d, gz.y / d);
                    gd_b[p] = -(gz.x * z.x + gz.y * z.y) / d;
                } else {
                    gn_b[p] = make_float2(0.f, 0.f);
                    gd_b[p] = 0.f;
                }
            }
#pragma unroll
            for (int c = 0; c < M; ++c) gWs[r][c] = nw[c];
            gq_b = dsv[r][r] > 0.f ? -0.5f * sr * sr * sr * gsv : 0.f;
        }
        __syncthreads();
        const float sr = ssv[r], gq = gq_b, invJ = 1.f / (float)J;
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = tid + f * NT;
            if (j >= J) continue;
            const float2 yr = yw[r][f];
            const float yr2 = abs2(yr);
            float2 ng = make_float2(sr * gy[r][f].x, sr * gy[r][f].y);
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                const float ph = phi(p, j);
                const float2 gn = gn_b[p];
                const float gd = gd_b[p];
                const float2 u = cmulf(conjf2(zs[r][p]), gy[p][f]);
                const float2 w = cmulf(conjf2(gn), yw[p][f]);
                ng = make_float2(ng.x - u.x + ph * w.x + 2.f * gd * ph * yr.x,
                                 ng.y - u.y + ph * w.y + 2.f * gd * ph * yr.y);
                const float2 t = cmul_conj(w, yr);       // conj(gn) y_p conj(y_r)
                gph[p][f] += t.x + gd * yr2;
            }
            const float phr = phi(r, j);
            ng = make_float2(ng.x + 2.f * invJ * gq * phr * yr.x, ng.y + 2.f * invJ * gq * phr * yr.y);
            gph[r][f] += gq * invJ * yr2;
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                const float ph = phi(p, j);
                const float2 t = cmulf(gn_b[p], yr);
                gy[p][f] = make_float2(gy[p][f].x + ph * t.x, gy[p][f].y + ph * t.y);
            }
            gy[r][f] = ng;
        }
    }

    // ---- outputs: dL/dY, dL/dW of the iteration start; eas: the warps' parts of
    // sum_j Re(conj(dL/dY) Y) (the sigma sums of the iteration before, completed at the end)
    {
        float ea[M];
        float2* gYo = g.gY + ((size_t)sm * F + i) * M * Jp;
#pragma unroll
        for (int r = 0; r < M; ++r) {
            ea[r] = 0.f;
#pragma unroll
            for (int f = 0; f < FPT; ++f) {
                const int j = tid + f * NT;
                if (j < J) {
                    const float2 y = y0s[r * Jp + j];
                    ea[r] = fmaf(gy[r][f].x, y.x, fmaf(gy[r][f].y, y.y, ea[r]));
                }
                if (j < Jp) gYo[(size_t)r * Jp + j] = j < J ? gy[r][f] : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int r = 0; r < M; ++r) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ea[r] += __shfl_xor_sync(0xffffffffu, ea[r], o);
            if (lane == 0) eas[(tid >> 5) * M + r] = ea[r];
        }
        if (tid < M * M) {
            const int p = tid / M, c = tid - p * M;
            g.gW[(((size_t)sm * F + i) * M + p) * M + c] = gWs[p][c];
        }
    }
    // ISS part of dL/dlambda: phi_r(j) = 1/lambda_{n, j-l} => dL/dlambda -= dL/dphi phi^2.
    // For one tap l every (n, j - l) target belongs to one thread.
    int lmax = 0;
    for (int n = 0; n < N; ++n) lmax = max(lmax, s.Ln[n]);
    for (int l = 0; l < lmax; ++l) {
        __syncthreads();
#pragma unroll
        for (int r = 0; r < M; ++r) {
            if (s.row_l[r] != l) continue;
            const int n = s.row_n[r];
#pragma unroll
            for (int f = 0; f < FPT; ++f) {
                const int j = tid + f * NT;
                if (j >= l && j < J) {
                    const float ph = invl[n * Jp + j - l];
                    gl[n * Jp + j - l] -= gph[r][f] * ph * ph;
                }
            }
        }
    }
    __syncthreads();
    // ---- lambda = T V: dL/dT += sum_j dL/dlambda V (this bin); the V part goes to kernel D
    for (int n = 0; n < N; ++n) {
        const float* Vn = Vsrc + (size_t)n * B * Jp;
        float gv[FPT];
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = tid + f * NT;
            float v = 0.f;
            if (j < J) v = invl[n * Jp + j] < thr ? gl[n * Jp + j] : 0.f;   // 0 where lambda is floored
            gv[f] = v;
            if (j < Jp) g.glt[((fb + n) * F + i) * (size_t)Jp + j] = v;
        }
        for (int kb = 0; kb < B; kb += 8) {
            float a[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) a[v] = 0.f;
#pragma unroll
            for (int f = 0; f < FPT; ++f) {
                const int j = tid + f * NT;
                if (j < J) {
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk)
                        if (kb + kk < B) a[kk] = fmaf(gv[f], Vn[(size_t)(kb + kk) * Jp + j], a[kk]);
                }
            }
            reduce_scatter<8>(a, lane);
            if (!(lane & 3) && kb + (lane >> 2) < B) atomicAdd(&gTacc[n * B + kb + (lane >> 2)], a[0]);
        }
    }
    __syncthreads();
    for (int t = tid; t < N * B; t += NT) {
        const int n = t / B, k = t - n * B;
        g.gT[tb + (size_t)n * FBp + (size_t)i * B + k] = gTacc[t];
    }
    // ---- the sigma sums of the iteration before this one (whose result is this iteration's
    // start state and dL/d of it the outputs above): e_r = sum_j Re(conj(dL/dY) Y)
    // + sum_c Re(conj(dL/dW) W) + [r = (n, 0)] 2 sum_k dL/dT T
    {
        float a[M];
#pragma unroll
        for (int r = 0; r < M; ++r) a[r] = tid < (NT >> 5) ? eas[tid * M + r] : 0.f;
        if (tid < M * M) {
            const int p = tid / M, c = tid - p * M;
            const float w = gWs[p][c].x * Wv[0][p][c].x + gWs[p][c].y * Wv[0][p][c].y;
#pragma unroll
            for (int r = 0; r < M; ++r)
                if (r == p) a[r] += w;
        }
        for (int t = tid; t < N * B; t += NT) {
            const int r0 = s.row0[t / B];
            const float v = 2.f * gTacc[t] * Ti[t];
#pragma unroll
            for (int r = 0; r < M; ++r)
                if (r == r0) a[r] += v;
        }
        block_sum<M>(a, red, bout);
        if (tid < M) atomicAdd(&g.e_prev[sm * M + tid], (double)bout[tid]);
    }
}

// ---------------------------------------------------------------- host templates
// Frames per thread of the per-bin adjoint: the fewest that keep the block at <= 256
// threads (cheaper block reductions, more independent loads per thread), else 4 frames
// with up to 512 threads.
inline int pick_fpt(int Jp, int* nt)
{
    for (int lim = 256; lim <= 512; lim += 256)
        for (int fpt = 1; fpt <= 4; fpt *= 2) {
            const int t = ((Jp + fpt - 1) / fpt + 31) / 32 * 32;
            if (t <= lim) {
                *nt = t < 64 ? 64 : t;
                return fpt;
            }
        }
    return 0;
}

inline size_t bin_smem(const Shape& s, bool vstage)
{
    return sizeof(float) * (size_t)(3 * s.N + 3 * s.M + (vstage ? s.N * s.B : 0)) * s.Jp;
}

// Stage V in shared memory when the block then still fits three to an SM.
inline bool stage_v(const Shape& s) { return bin_smem(s, true) <= 64 * 1024; }


template <int M, int FPT>
cudaError_t bin_mf(const Shape& s, int S, const StatePtrs* cur, const StatePtrs* nxt, const GradBufs& g, int nt,
                   cudaStream_t st, bool configure)
{
    const bool vs = stage_v(s);
    const size_t smem = bin_smem(s, vs);
    if (configure) return cudaFuncSetAttribute(grad_bin_kernel<M, FPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    grad_bin_kernel<M, FPT><<<dim3(s.F, S), nt, smem, st>>>(s, cur, nxt, g, vs ? 1 : 0);
    return cudaGetLastError();
}

template <int M>
inline cudaError_t bin_m(const Shape& s, int S, const StatePtrs* cur, const StatePtrs* nxt, const GradBufs& g,
                  cudaStream_t st, bool configure)
{
    int nt = 0;
    switch (pick_fpt(s.Jp, &nt)) {
        case 1: return bin_mf<M, 1>(s, S, cur, nxt, g, nt, st, configure);
        case 2: return bin_mf<M, 2>(s, S, cur, nxt, g, nt, st, configure);
        case 4: return bin_mf<M, 4>(s, S, cur, nxt, g, nt, st, configure);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ctf
