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

template <int M, int FPT>
__global__ void __launch_bounds__(512)
bin_phase_kernel(const Shape s, const State d, const int v_tap0)
{
    extern __shared__ float smem[];
    const int i = blockIdx.x;
    const int NT = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
    const int J = s.J, Jp = s.Jp, N = s.N, B = s.B;

    float* sq = smem;                    // [M][Jp]  |y_r(j)|^2 after the sweep
    float* Aw = sq + M * Jp;             // [N][Jp]  P_n(j) / lambda^2
    float* Cw = Aw + N * Jp;             // [N][Jp]  c_n(j) / lambda
    float* red = Cw + N * Jp;            // [2][NW][3M] per-warp partial sums

    float scl[M];
#pragma unroll
    for (int r = 0; r < M; ++r) scl[r] = d.scale[r];

    // ---- load y (with the pending scale) and the delayed weights
    const float2* Yb = d.Y + (size_t)i * M * Jp;
    const float* il = d.invlam + (size_t)i * N * Jp;
    float2 y[M][FPT];
    float phi[M][FPT];
#pragma unroll
    for (int r = 0; r < M; ++r) {
        const int n = s.row_n[r], l = s.row_l[r];
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int j = tid + f * NT;
            float2 v = make_float2(0.f, 0.f);
            float w = 0.f;
            if (j < J) {
                v = Yb[(size_t)r * Jp + j];
                v.x *= scl[r];
                v.y *= scl[r];
                if (j >= l) w = il[(size_t)n * Jp + j - l];
            }
            y[r][f] = v;
            phi[r][f] = w;
        }
    }

    // thread m < M keeps column m of W_i
    float2 wcol[M];
    if (tid < M) {
#pragma unroll
        for (int p = 0; p < M; ++p) {
            float2 w = d.W[((size_t)i * M + p) * M + tid];
            wcol[p] = make_float2(w.x * scl[p], w.y * scl[p]);
        }
    }

    double dlog = 0.0;
    // ---- ISS sweep
#pragma unroll
    for (int r = 0; r < M; ++r) {
        float acc[3 * M];
#pragma unroll
        for (int k = 0; k < 3 * M; ++k) acc[k] = 0.f;
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const float2 yr = y[r][f];
            const float pr = abs2(yr);
#pragma unroll
            for (int p = 0; p < M; ++p) {
                acc[p] = fmaf(phi[p][f], pr, acc[p]);
                if (p != r) {
                    const float2 c = cmul_conj(y[p][f], yr);
                    acc[M + 2 * p] = fmaf(phi[p][f], c.x, acc[M + 2 * p]);
                    acc[M + 2 * p + 1] = fmaf(phi[p][f], c.y, acc[M + 2 * p + 1]);
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
        const double q = (double)tot[r] / (double)J;
        float sc = 1.0f;
        if (q > 0.0) {
            const double scd = 1.0 / sqrt(q);
            sc = (float)scd;
            dlog += -0.5 * log(q);
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

    // ---- store y, W, log|det W|; stage |y|^2
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
    if (tid == 0) {
        double ls = 0.0;
#pragma unroll
        for (int r = 0; r < M; ++r) ls += log((double)scl[r]);
        d.logdet[i] += ls + dlog;
    }
    __syncthreads();

    // ---- delayed power and the basis-update weights at this thread's frames
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
            const float w = phi[p][f];          // 1/lambda_{n,i,j} (tap 0 has no delay)
            Aw[n * Jp + j] = P * w * w;
            Cw[n * Jp + j] = cnt * w;
            Pout[(size_t)n * Jp + j] = v_tap0 ? sq[p * Jp + j] : P;
        }
    }
    __syncthreads();

    // ---- basis MU (one warp per (n,k)) and per-row power sums for mu
    const int npairs = N * B;
    for (int t = warp; t < npairs + M; t += NW) {
        if (t < npairs) {
            const int n = t / B, k = t - n * B;
            const float* Vk = d.V + (size_t)(n * B + k) * Jp;
            const float* An = Aw + n * Jp;
            const float* Cn = Cw + n * Jp;
            float a = 0.f, c = 0.f;
            for (int j = lane; j < J; j += 32) {
                const float v = Vk[j];
                a = fmaf(v, An[j], a);
                c = fmaf(v, Cn[j], c);
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
            float a = 0.f;
            for (int j = lane; j < J; j += 32) a += sq[r * Jp + j];
            a = warp_sum(a);
            if (lane == 0) d.mupart[(size_t)i * M + r] = a;
        }
    }
}

bool bin_phase_config(int M, int J, int* fpt, int* threads)
{
    static const int cands[4] = {1, 2, 4, 8};
    // prefer about 256 threads; fall back to 512 for the longest frames
    for (int pass = 0; pass < 2; ++pass) {
        const int cap = pass == 0 ? 256 : 512;
        for (int c = 0; c < 4; ++c) {
            const int f = cands[c];
            if (M * f > 32) break;
            const int nt = (J + f - 1) / f;
            if (nt <= cap) {
                *fpt = f;
                *threads = ((nt + 31) / 32) * 32;
                if (*threads < 64) *threads = 64;
                return true;
            }
        }
    }
    return false;
}

size_t bin_phase_smem(const Shape& s)
{
    int fpt = 0, nt = 0;
    bin_phase_config(s.M, s.J, &fpt, &nt);
    const int NW = nt / 32;
    return sizeof(float) * ((size_t)(s.M + 2 * s.N) * s.Jp + 2 * NW * 3 * s.M);
}

template <int M, int FPT>
static cudaError_t launch_mf(const Shape& s, const State& d, int v_tap0, int nt, cudaStream_t st,
                            bool configure_only)
{
    if (configure_only) {
        // the device's opt-in maximum, so that handles of different J share the setting
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        if ((size_t)optin < bin_phase_smem(s)) return cudaErrorInvalidValue;
        return cudaFuncSetAttribute(bin_phase_kernel<M, FPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    }
    bin_phase_kernel<M, FPT><<<s.F, nt, bin_phase_smem(s), st>>>(s, d, v_tap0);
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
