// Bin phase of one CTF-MNMF-ISS iteration: one CTA per frequency bin.
//
// Per bin i (Sec. III):
//   0. apply the pending normalisation of the previous iteration (Eqs. 19-21):
//      y_r *= s_r, row r of W *= s_r, T[n] *= s_{(n,0)}^2, log|det W| += sum log s_r
//   1. frame weights phi_r(j) = 1/lambda_{n(r),i,j-l(r)} for j >= l(r), else 0 (Eq. 8)
//   2. ISS sweep, r = 0..M-1 in order (Eqs. 11-16), on the data-domain form
//        w_p^H Q_p w_r = (1/J) sum_j phi_p(j) y_p(j) conj(y_r(j)),
//        z_p = sum_j phi_p y_p conj(y_r) / sum_j phi_p |y_r|^2           (p != r)
//        z_r = 1 - q^{-1/2},  q = (1/J) sum_j phi_r |y_r|^2   (q, q^{-1/2}, log q in FP64)
//        y_p <- y_p - z_p y_r,  W_i <- W_i - z w_r^H,  log|det W_i| += log|1 - z_r| (lemma)
//   3. basis MU (Eq. 17): T[n,i,k] <- T sqrt( sum_j V[n,k,j] P_n(j)/lambda^2 / sum_j V c_n(j)/lambda ),
//      P_n(j) = sum_{l < L_n, j+l < J} |y_{(n,l)}(j+l)|^2, c_n(j) = #{l < L_n : j+l < J}
//   4. outputs for the cross-bin steps: P (or |y_{(n,0)}|^2 for the tap-0 activation
//      update) and the per-bin row powers sum_j |y_r|^2 for mu_r.
//
// The bin's M x J samples live in registers (thread t owns frames t, t+NT, ...); the
// J-reductions are warp shuffles plus one shared-memory pass per ISS step.
#include "internal.cuh"

namespace ctf {

constexpr int kLPad = 8;   // zero frames in front of each staged 1/lambda row (taps <= 8)

template <int M, int FPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
bin_phase_kernel(const Shape s, const State d, const int v_tap0)
{
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const int i = blockIdx.x;
    const int NT = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
    const int J = s.J, Jp = s.Jp, N = s.N, B = s.B;
    const int LR = kLPad + Jp;           // staged row length

    float* ils = smem;                   // [N][LR] 1/lambda_{n,i,j} at kLPad + j, zeros in front;
                                         //         reused for P_n(j)/lambda^2 after the sweep
    float* Cw = ils + N * LR;            // [N][Jp]  c_n(j) / lambda
    float* sq = Cw + N * Jp;             // [M][Jp]  |y_r(j)|^2 after the sweep
    float* red = sq + M * Jp;            // [2][NW][3M] per-warp partial sums

    // ---- stage 1/lambda of this bin (float4, coalesced; the front pad is zero)
    {
        const float4* src = reinterpret_cast<const float4*>(d.invlam + (size_t)i * N * Jp);
        const int LR4 = LR >> 2, J4 = Jp >> 2, P4 = kLPad >> 2;
        for (int e = tid; e < N * LR4; e += NT) {
            const int n = e / LR4, o = e - n * LR4;
            smem4[e] = (o < P4) ? make_float4(0.f, 0.f, 0.f, 0.f) : src[(size_t)n * J4 + o - P4];
        }
    }

    float scl[M];
#pragma unroll
    for (int r = 0; r < M; ++r) scl[r] = d.scale[r];

    // ---- load y with the pending scale (padding frames are zero in memory)
    const float2* Yb = d.Y + (size_t)i * M * Jp;
    float2 y[M][FPT];
#pragma unroll
    for (int r = 0; r < M; ++r) {
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = tid + f * NT;
            float2 v = make_float2(0.f, 0.f);
            if (j < Jp) v = Yb[(size_t)r * Jp + j];
            y[r][f] = make_float2(v.x * scl[r], v.y * scl[r]);
        }
    }

    // thread m < M keeps column m of W_i
    float2 wcol[M];
    if (tid < M) {
#pragma unroll
        for (int p = 0; p < M; ++p) {
            const float2 w = d.W[((size_t)i * M + p) * M + tid];
            wcol[p] = make_float2(w.x * scl[p], w.y * scl[p]);
        }
    }
    __syncthreads();

    double qprod = 1.0;                  // product of the q_r of the sweep (thread 0)
    const float invJ = 1.0f / (float)J;
    // ---- ISS sweep
#pragma unroll
    for (int r = 0; r < M; ++r) {
        float acc[3 * M];
#pragma unroll
        for (int k = 0; k < 3 * M; ++k) acc[k] = 0.f;
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = min(tid + f * NT, Jp - 1);   // frames past Jp hold y = 0
            const float2 yr = y[r][f];
            const float pr = abs2(yr);
#pragma unroll
            for (int p = 0; p < M; ++p) {
                const float ph = ils[s.row_n[p] * LR + kLPad + j - s.row_l[p]];
                acc[p] = fmaf(ph, pr, acc[p]);
                if (p != r) {
                    const float2 c = cmul_conj(y[p][f], yr);
                    acc[M + 2 * p] = fmaf(ph, c.x, acc[M + 2 * p]);
                    acc[M + 2 * p + 1] = fmaf(ph, c.y, acc[M + 2 * p + 1]);
                }
            }
        }
        float* rb = red + (r & 1) * NW * 3 * M;
#pragma unroll
        for (int k = 0; k < 3 * M; ++k) {
            if (k >= M && (k - M) / 2 == r) continue;
            const float v = warp_sum(acc[k]);
            if (lane == 0) rb[warp * 3 * M + k] = v;
        }
        __syncthreads();
        float tot[3 * M];
#pragma unroll
        for (int k = 0; k < 3 * M; ++k) tot[k] = 0.f;
        for (int w = 0; w < NW; ++w) {
#pragma unroll
            for (int k = 0; k < 3 * M; ++k) {
                if (k >= M && (k - M) / 2 == r) continue;
                tot[k] += rb[w * 3 * M + k];
            }
        }
        float2 z[M];
#pragma unroll
        for (int p = 0; p < M; ++p) {
            z[p] = make_float2(0.f, 0.f);
            if (p != r && tot[p] > 0.f) {
                const float inv = 1.0f / tot[p];
                z[p] = make_float2(tot[M + 2 * p] * inv, tot[M + 2 * p + 1] * inv);
            }
        }
        // q = (1/J) sum_j phi_r |y_r|^2; 1 - z_r = q^{-1/2} (FP32 reciprocal square root with
        // one Newton step); log|1 - z_r| is accumulated in FP64 through the product of q.
        const float q = tot[r] * invJ;
        float sc = 1.0f;
        if (q > 0.f) {
            const float r0 = rsqrtf(q);
            sc = r0 * fmaf(-0.5f * q * r0, r0, 1.5f);
            if (tid == 0) qprod *= (double)q;
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
            y[r][f] = make_float2(yr.x * sc, yr.y * sc);
        }
        if (tid < M) {
            const float2 wr = wcol[r];
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p == r) continue;
                wcol[p].x -= z[p].x * wr.x - z[p].y * wr.y;
                wcol[p].y -= z[p].x * wr.y + z[p].y * wr.x;
            }
            wcol[r] = make_float2(wr.x * sc, wr.y * sc);
        }
    }

    // ---- store y and W; stage |y|^2
    float2* Yo = d.Y + (size_t)i * M * Jp;
#pragma unroll
    for (int r = 0; r < M; ++r) {
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = tid + f * NT;
            if (j < Jp) {
                Yo[(size_t)r * Jp + j] = y[r][f];
                sq[r * Jp + j] = abs2(y[r][f]);
            }
        }
    }
    if (tid < M) {
#pragma unroll
        for (int p = 0; p < M; ++p) d.W[((size_t)i * M + p) * M + tid] = wcol[p];
    }
    __syncthreads();

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
            const int j = tid + f * NT;
            if (j >= Jp) continue;
            float P = 0.f, cnt = 0.f;
            if (j < J) {
                for (int l = 0; l < Lp && j + l < J; ++l) {
                    P += sq[(p + l) * Jp + j + l];
                    cnt += 1.f;
                }
            }
            float* wp = ils + n * LR + kLPad + j;
            const float w = *wp;                // 1/lambda_{n,i,j} (zero past J)
            *wp = P * w * w;
            Cw[n * Jp + j] = cnt * w;
            Pout[(size_t)n * Jp + j] = v_tap0 ? sq[p * Jp + j] : P;
        }
    }
    __syncthreads();

    // ---- basis MU: one warp per (n,k); V rows through the L1 (shared by the CTAs of an
    //      SM), float4, a batch of independent loads per lane before the FMAs
    const int npairs = N * B;
    const int J4 = Jp >> 2;
    for (int t = warp; t < npairs + M; t += NW) {
        if (t < npairs) {
            const int n = t / B, k = t - n * B;
            const float4* V4 = reinterpret_cast<const float4*>(d.V + (size_t)(n * B + k) * Jp);
            const float4* A4 = reinterpret_cast<const float4*>(ils + n * LR + kLPad);
            const float4* C4 = reinterpret_cast<const float4*>(Cw + n * Jp);
            float a = 0.f, c = 0.f;
            for (int base = lane; base < J4; base += 32 * 8) {
                float4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int q = base + 32 * u;
                    v[u] = q < J4 ? __ldg(V4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int q = base + 32 * u;
                    if (q < J4) {
                        const float4 x = A4[q], cc = C4[q];
                        a = fmaf(v[u].x, x.x, fmaf(v[u].y, x.y, fmaf(v[u].z, x.z, fmaf(v[u].w, x.w, a))));
                        c = fmaf(v[u].x, cc.x, fmaf(v[u].y, cc.y, fmaf(v[u].z, cc.z, fmaf(v[u].w, cc.w, c))));
                    }
                }
            }
            a = warp_sum(a);
            c = warp_sum(c);
            if (lane == 0) {
                const float s0 = d.scale[s.row0[n]];
                float* Tp = d.T + ((size_t)i * N + n) * B + k;
                const float tcur = *Tp * (s0 * s0);
                float tn = (c > 0.f) ? tcur * sqrtf(a / c) : tcur;
                *Tp = fmaxf(tn, kFloorNmf);
            }
        } else {
            const int r = t - npairs;
            const float4* S4 = reinterpret_cast<const float4*>(sq + r * Jp);
            float a = 0.f;
            for (int q = lane; q < J4; q += 32) {
                const float4 x = S4[q];
                a += (x.x + x.y) + (x.z + x.w);
            }
            a = warp_sum(a);
            if (lane == 0) d.mupart[(size_t)i * M + r] = a;
        }
    }

    // ---- log|det W_i| (FP64): pending scale and the sweep, log|1 - z_r| = -log(q_r)/2
    if (tid == 0) {
        double sp = 1.0;
#pragma unroll
        for (int r = 0; r < M; ++r) sp *= (double)scl[r];
        d.logdet[i] += log(sp) - 0.5 * log(qprod);
    }
}

bool bin_phase_config(int M, int J, int* fpt, int* threads)
{
    // frames per thread 1, 2, 4 with at most 256 threads; 8 (M <= 4) with up to 512
    static const int cands[4] = {1, 2, 4, 8};
    for (int c = 0; c < 4; ++c) {
        const int f = cands[c];
        if (M * f > 32) break;
        const int cap = f == 8 ? 512 : 256;
        const int nt = (J + f - 1) / f;
        if (nt <= cap) {
            *fpt = f;
            *threads = ((nt + 31) / 32) * 32;
            if (*threads < 64) *threads = 64;
            return true;
        }
    }
    return false;
}

size_t bin_phase_smem(const Shape& s)
{
    int fpt = 0, nt = 0;
    bin_phase_config(s.M, s.J, &fpt, &nt);
    const int NW = nt / 32;
    return sizeof(float) * ((size_t)s.N * (kLPad + s.Jp) + (size_t)(s.N + s.M) * s.Jp + 2 * NW * 3 * s.M);
}

template <int M, int FPT>
static cudaError_t launch_mf(const Shape& s, const State& d, int v_tap0, int nt, cudaStream_t st,
                            bool configure_only)
{
    // 8 frames per thread: up to 512 threads, 128 registers; otherwise 256 threads and
    // 4 CTAs per SM (64 registers) when the bin's samples take at most 24 registers
    constexpr int kMaxT = FPT == 8 ? 512 : 256;
    constexpr int kMinB = FPT == 8 ? 1 : (M * FPT >= 16 ? 2 : 4);
    if (configure_only) {
        // the device's opt-in maximum, so that handles of different J share the setting
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        if ((size_t)optin < bin_phase_smem(s)) return cudaErrorInvalidValue;
        return cudaFuncSetAttribute(bin_phase_kernel<M, FPT, kMaxT, kMinB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    }
    // float4 views of the staged rows need 16-byte aligned row starts
    if (s.Jp % 8 != 0 || nt > kMaxT) return cudaErrorInvalidValue;
    bin_phase_kernel<M, FPT, kMaxT, kMinB><<<s.F, nt, bin_phase_smem(s), st>>>(s, d, v_tap0);
    return cudaGetLastError();
}

template <int M>
static cudaError_t launch_m(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st,
                           bool cfg)
{
    switch (fpt) {
        case 1: return launch_mf<M, 1>(s, d, v_tap0, nt, st, cfg);
        case 2: return launch_mf<M, 2>(s, d, v_tap0, nt, st, cfg);
        case 4: return launch_mf<M, 4>(s, d, v_tap0, nt, st, cfg);
        case 8: if constexpr (M <= 4) return launch_mf<M, 8>(s, d, v_tap0, nt, st, cfg);
                return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

static cudaError_t dispatch(const Shape& s, const State& d, int v_tap0, cudaStream_t st, bool cfg)
{
    int fpt = 0, nt = 0;
    if (!bin_phase_config(s.M, s.J, &fpt, &nt)) return cudaErrorInvalidValue;
    switch (s.M) {
        case 2: return launch_m<2>(s, d, v_tap0, fpt, nt, st, cfg);
        case 3: return launch_m<3>(s, d, v_tap0, fpt, nt, st, cfg);
        case 4: return launch_m<4>(s, d, v_tap0, fpt, nt, st, cfg);
        case 5: return launch_m<5>(s, d, v_tap0, fpt, nt, st, cfg);
        case 6: return launch_m<6>(s, d, v_tap0, fpt, nt, st, cfg);
        case 7: return launch_m<7>(s, d, v_tap0, fpt, nt, st, cfg);
        case 8: return launch_m<8>(s, d, v_tap0, fpt, nt, st, cfg);
    }
    return cudaErrorInvalidValue;
}

// Raise the dynamic shared-memory limit of the instantiation this shape uses (once per
// handle, outside any stream capture).
cudaError_t configure_bin_phase(const Shape& s)
{
    State none = {};
    return dispatch(s, none, 0, nullptr, true);
}

cudaError_t launch_bin_phase(const Shape& s, const State& d, int v_tap0, cudaStream_t st)
{
    return dispatch(s, d, v_tap0, st, false);
}

}  // namespace ctf
