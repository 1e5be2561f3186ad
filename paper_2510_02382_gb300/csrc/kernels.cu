// Kernels of libctfmnmf other than the bin phase: loading, NMF initialisation, the
// source PSD, the cross-bin activation update with normalisation, the cost, the
// source images and the read-outs.
#include <math.h>

#include "phases.cuh"

namespace ctf {

// ------------------------------------------------------------------ load (Sec. V-A init)
// Y[i][m][j] = X[m][i][j] (W_i = I so y = x), zero padding frames; W = I, log|det| = 0,
// pending scale 1. flag[0] is set if X holds a non-finite value.
__global__ void load_kernel(const Shape s, const State d, const float2* __restrict__ X)
{
    const int i = blockIdx.x, m = blockIdx.y;
    const int M = s.M, F = s.F, J = s.J, Jp = s.Jp;
    const float2* src = X + ((size_t)m * F + i) * J;
    float2* dst = d.Y + ((size_t)i * M + m) * Jp;
    bool bad = false;
    for (int j = threadIdx.x; j < Jp; j += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (j < J) {
            v = src[j];
            bad |= !(isfinite(v.x) && isfinite(v.y));
        }
        dst[j] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(d.flag, 1);
    if (threadIdx.x < M) d.W[((size_t)i * M + m) * M + threadIdx.x] = make_float2(m == (int)threadIdx.x ? 1.f : 0.f, 0.f);
    if (m == 0 && threadIdx.x == 0) {
        d.logdet[i] = 0.0;
        d.ldm[i] = 1.0;
        d.lde[i] = 0;
    }
    if (i == 0 && m == 0 && threadIdx.x < M) d.scale[threadIdx.x] = 1.f;
}

cudaError_t launch_load(const Shape& s, const State& d, const float2* X, cudaStream_t st)
{
    load_kernel<<<dim3(s.F, s.M), 256, 0, st>>>(s, d, X);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ NMF factors
// Default values: splitmix64 (Steele, Lea, Flood 2014; the constants of Vigna's
// public-domain splitmix64.c) of the counter seed*2^32 + c, top 24 bits as u in [0,1).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float default_factor(uint64_t seed, uint64_t c)
{
    const double u = (double)(splitmix64((seed << 32) + c) >> 40) * (1.0 / 16777216.0);
    return (float)(0.1 + 0.9 * u);
}

// Probe state for timing the two execution paths: rows with pseudo-random entries in
// (-1/2, 1/2) + i(-1/2, 1/2) from the splitmix64 counter hash, zero padding frames, W = I,
// log|det| = 0, no pending scale.
__global__ void probe_fill_kernel(const Shape s, const State d)
{
    const int i = blockIdx.x, m = blockIdx.y;
    const int M = s.M, J = s.J, Jp = s.Jp;
    float2* dst = d.Y + ((size_t)i * M + m) * Jp;
    for (int j = threadIdx.x; j < Jp; j += blockDim.x) {
        const uint64_t c = ((uint64_t)i * M + m) * (uint64_t)Jp + j;
        const uint64_t h = splitmix64(0x5eedull * 0x100000000ull + c);
        const float re = (float)(h >> 40) * (1.0f / 16777216.0f) - 0.5f;
        const float im = (float)((h >> 16) & 0xffffff) * (1.0f / 16777216.0f) - 0.5f;
        dst[j] = j < J ? make_float2(re, im) : make_float2(0.f, 0.f);
    }
    if ((int)threadIdx.x < M) d.W[((size_t)i * M + m) * M + threadIdx.x] = make_float2(m == (int)threadIdx.x ? 1.f : 0.f, 0.f);
    if (m == 0 && threadIdx.x == 0) {
        d.logdet[i] = 0.0;
        d.ldm[i] = 1.0;
        d.lde[i] = 0;
    }
    if (i == 0 && m == 0 && (int)threadIdx.x < M) d.scale[threadIdx.x] = 1.f;
}

cudaError_t launch_probe_fill(const Shape& s, const State& d, cudaStream_t st)
{
    probe_fill_kernel<<<dim3(s.F, s.M), 256, 0, st>>>(s, d);
    return cudaGetLastError();
}

// T0 [N][F][B] -> T [F][N][B]; V0 [N][B][J] -> V [N][B][Jp]. Null source: keep, or the
// default init when `use_default` is set.
__global__ void init_nmf_kernel(const Shape s, const State d, const float* __restrict__ T0,
                                const float* __restrict__ V0, int use_default, uint64_t seed)
{
    const int N = s.N, F = s.F, B = s.B, J = s.J, Jp = s.Jp;
    const size_t nT = (size_t)N * F * B, nV = (size_t)N * B * Jp;
    bool bad = false;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nT + nV;
         e += (size_t)gridDim.x * blockDim.x) {
        if (e < nT) {
            // e is the flat index of T0[n][i][k]
            const int k = (int)(e % B);
            const int i = (int)((e / B) % F);
            const int n = (int)(e / ((size_t)B * F));
            float v;
            if (T0) v = T0[e];
            else if (use_default) v = default_factor(seed, 2 * e);
            else continue;
            bad |= !isfinite(v);
            d.T[(size_t)n * s.FBp + (size_t)i * B + k] = fmaxf(v, s.floor_nmf);
        } else {
            const size_t f = e - nT;               // index into V [N][B][Jp]
            const int j = (int)(f % Jp);
            const size_t nk = f / Jp;
            float v = 0.f;
            if (j < J) {
                const size_t src = nk * J + j;     // flat index of V0[n][k][j]
                if (V0) v = V0[src];
                else if (use_default) v = default_factor(seed, 2 * src + 1);
                else continue;
                bad |= !isfinite(v);
                v = fmaxf(v, s.floor_nmf);
            }
            d.V[f] = v;
        }
    }
    if (bad) atomicOr(d.flag, 2);
}

cudaError_t launch_init_nmf(const Shape& s, const State& d, const float* T0, const float* V0,
                            uint64_t seed, cudaStream_t st)
{
    const int use_default = (T0 == nullptr && V0 == nullptr) ? 1 : 0;
    init_nmf_kernel<<<256, 256, 0, st>>>(s, d, T0, V0, use_default, seed);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ source PSD
// invlam[i][n][j] = 1 / max(sum_k T[i][n][k] V[n][k][j], floor) (Sec. II NMF model).
__global__ void psd_kernel(const Shape s, const State d)
{
    const int N = s.N, F = s.F, B = s.B, J = s.J, Jp = s.Jp;
    const size_t total = (size_t)F * N * Jp;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % Jp);
        const size_t in = e / Jp;
        const int n = (int)(in % N);
        const int i = (int)(in / N);
        float out = 0.f;
        if (j < J) {
            const float* Ti = d.T + (size_t)n * s.FBp + (size_t)i * B;
            float lam = 0.f;
            for (int k = 0; k < B; ++k) lam = fmaf(Ti[k], d.V[((size_t)n * B + k) * Jp + j], lam);
            out = recip(fmaxf(lam, kFloorPsd));
        }
        d.invlam[e] = out;
    }
}

cudaError_t launch_psd(const Shape& s, const State& d, cudaStream_t st)
{
    psd_kernel<<<1024, 256, 0, st>>>(s, d);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ frame phase
// Two-kernel path: blocks 0 .. kFoldBlocks-1 fold the bin phase's |det| factors into the FP64
// log-det pairs, one bin per thread (FP64 is slow on this GPU, so no single block takes all
// bins); block 0 also forms the normalisation scale of this iteration from the per-bin row
// powers (FP64, Eq. 19) and stores it as the pending scale of the next bin phase; every other
// block (256 threads) takes one (8-frame tile, source) item, whose device code is
// frame_item() in phases.cuh (the items need no scale: the next bin phase applies it).
constexpr int kFrameThreads = 256;
constexpr int kFoldBlocks = 8;
constexpr int kFrameSmemBytes = 48 * 1024;

// EXACT: s.B equals the class width BB (the per-basis bounds tests fold away).
template <int BB, bool EXACT>
__global__ void __launch_bounds__(kFrameThreads) frame_phase_kernel(const Shape s, const State d,
                                                                    const int v_tap0, const int normalize,
                                                                    const int FC)
{
    extern __shared__ float4 fsm4[];
#ifdef CTFMNMF_DEBUG
    if ((int)blockIdx.x >= (s.Jp / kFrameTile) * s.N + kFoldBlocks) {     // an item outside the shape
        if (threadIdx.x == 0) atomicOr(d.flag + 3, 1);
        return;
    }
#endif
    if (blockIdx.x < kFoldBlocks) {
        fold_logdet(s, d, blockIdx.x * kFrameThreads + threadIdx.x, kFoldBlocks * kFrameThreads);
        if (blockIdx.x == 0) scales_fp64<false>(s, d, normalize, reinterpret_cast<double*>(fsm4));
        return;
    }
    const Grp g{(int)threadIdx.x, kFrameThreads, 0};
    const int item = blockIdx.x - kFoldBlocks;
    if constexpr (BB <= 16)
        frame_item<BB, EXACT, true>(s, d, item, g, reinterpret_cast<float*>(fsm4), FC, v_tap0);
    else
        frame_item_wide<BB, EXACT, true>(s, d, item, g, reinterpret_cast<float*>(fsm4), FC, v_tap0);
}

static int frame_fc(const Shape& s, int BB)
{
    const int fixed = BB == 4 ? frame_smem_fixed<4>(kFrameThreads)
                    : BB == 8 ? frame_smem_fixed<8>(kFrameThreads)
                    : BB == 10 ? frame_smem_fixed<10>(kFrameThreads)
                    : BB == 16 ? frame_smem_fixed<16>(kFrameThreads) : frame_smem_fixed<32>(kFrameThreads);
    return frame_chunk(kFrameSmemBytes / 4, s.B, fixed);
}

static int frame_bb(int B) { return B <= 4 ? 4 : B <= 8 ? 8 : B <= 10 ? 10 : B <= 16 ? 16 : 32; }

template <int BB>
static cudaError_t frame_bb_set(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(frame_phase_kernel<BB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(frame_phase_kernel<BB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

// Allow the frame-phase kernels more than 48 KB of shared memory (dynamic + static).
cudaError_t configure_frame_phase()
{
    const int bytes = kFrameSmemBytes;
    cudaError_t e = frame_bb_set<4>(bytes);
    if (e == cudaSuccess) e = frame_bb_set<8>(bytes);
    if (e == cudaSuccess) e = frame_bb_set<10>(bytes);
    if (e == cudaSuccess) e = frame_bb_set<16>(bytes);
    if (e == cudaSuccess) e = frame_bb_set<32>(bytes);
    return e;
}

template <int BB>
static void frame_launch(const Shape& s, const State& d, int v_tap0, int normalize, int FC, int items, size_t smem,
                         cudaStream_t st)
{
    if (s.B == BB) frame_phase_kernel<BB, true><<<items, kFrameThreads, smem, st>>>(s, d, v_tap0, normalize, FC);
    else frame_phase_kernel<BB, false><<<items, kFrameThreads, smem, st>>>(s, d, v_tap0, normalize, FC);
}

cudaError_t launch_frame_phase(const Shape& s, const State& d, int v_tap0, int normalize,
                               cudaStream_t st)
{
    const int items = (s.Jp / kFrameTile) * s.N + kFoldBlocks;   // + the fold and scale blocks
    const int BB = frame_bb(s.B);
    const int FC = frame_fc(s, BB);
    if (FC < 4 || (FC * s.B) % 4 != 0 || s.Jp % kFrameTile != 0) return cudaErrorInvalidValue;
    const size_t smem = kFrameSmemBytes;
    switch (BB) {
        case 4: frame_launch<4>(s, d, v_tap0, normalize, FC, items, smem, st); break;
        case 8: frame_launch<8>(s, d, v_tap0, normalize, FC, items, smem, st); break;
        case 10: frame_launch<10>(s, d, v_tap0, normalize, FC, items, smem, st); break;
        case 16: frame_launch<16>(s, d, v_tap0, normalize, FC, items, smem, st); break;
        default: frame_launch<32>(s, d, v_tap0, normalize, FC, items, smem, st); break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ finalize
// Apply the pending normalisation (scale) to Y rows, W rows, log|det|, T and the stored
// 1/lambda, after the last iteration of a call. One CTA per (bin, row).
__global__ void finalize_kernel(const Shape s, const State d)
{
    const int i = blockIdx.x, r = blockIdx.y;
    const int M = s.M, N = s.N, B = s.B, Jp = s.Jp;
    const float sc = d.scale[r];
    float2* row = d.Y + ((size_t)i * M + r) * Jp;
    for (int j = threadIdx.x; j < Jp; j += blockDim.x) {
        float2 v = row[j];
        row[j] = make_float2(v.x * sc, v.y * sc);
    }
    if (threadIdx.x < M) {
        float2* w = d.W + ((size_t)i * M + r) * M + threadIdx.x;
        *w = make_float2(w->x * sc, w->y * sc);
    }
    if (r == 0 && threadIdx.x == 0) {
        // fold the running |det| product and the pending row scales into log|det W_i|
        double f = d.ldm[i];
        for (int p = 0; p < M; ++p) f *= (double)d.scale[p];
        d.logdet[i] += log(f) + (double)d.lde[i] * 0.69314718055994530942;
        d.ldm[i] = 1.0;
        d.lde[i] = 0;
    }
    if (s.row_l[r] == 0) {
        const int n = s.row_n[r];
        if (threadIdx.x < B) d.T[(size_t)n * s.FBp + (size_t)i * B + threadIdx.x] *= sc * sc;
        float* il = d.invlam + ((size_t)i * s.N + n) * Jp;
        const float fac = 1.0f / (sc * sc);
        for (int j = threadIdx.x; j < Jp; j += blockDim.x) il[j] = scaled_invlam(il[j], fac);
    }
}

// ------------------------------------------------------------------ NaN/Inf scan
// Y [F][M][Jp] complex64, T [N][FBp] and V [N][B][Jp] float32: flag[2] is set if any value is
// not finite (ctfmnmf_options.check_finite, and every iteration of a CTFMNMF_DEBUG build).
__global__ void finite_scan_kernel(const Shape s, const State d)
{
    const size_t nY = (size_t)s.F * s.M * s.Jp * 2, nT = (size_t)s.N * s.FBp, nV = (size_t)s.N * s.B * s.Jp;
    const float* Yf = reinterpret_cast<const float*>(d.Y);
    bool bad = false;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nY + nT + nV;
         e += (size_t)gridDim.x * blockDim.x) {
        const float v = e < nY ? Yf[e] : e < nY + nT ? d.T[e - nY] : d.V[e - nY - nT];
        bad |= !isfinite(v);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(d.flag + 2, 1);
}

cudaError_t launch_finite_scan(const Shape& s, const State& d, cudaStream_t st)
{
    finite_scan_kernel<<<304, 256, 0, st>>>(s, d);
    return cudaGetLastError();
}

__global__ void reset_scale_kernel(const Shape s, const State d)
{
    if (threadIdx.x < s.M) d.scale[threadIdx.x] = 1.f;
}

cudaError_t launch_finalize(const Shape& s, const State& d, cudaStream_t st)
{
    finalize_kernel<<<dim3(s.F, s.M), 256, 0, st>>>(s, d);
    reset_scale_kernel<<<1, 32, 0, st>>>(s, d);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ cost (Eq. 5)
// Per bin: sum over rows r = (n,l) and frames j >= l of log lambda_{n,i,j-l} +
// |y_r(j)|^2 / lambda_{n,i,j-l} (FP32 terms, FP64 accumulation), minus 2 J log|det W_i|.
// Assumes no pending normalisation (ctfmnmf_iterate always ends with finalize).
__global__ void cost_bin_kernel(const Shape s, const State d)
{
    __shared__ double part[32];
    const int i = blockIdx.x;
    const int M = s.M, N = s.N, J = s.J, Jp = s.Jp;
    double acc = 0.0;
    for (int r = 0; r < M; ++r) {
        const int n = s.row_n[r], l = s.row_l[r];
        const float2* yr = d.Y + ((size_t)i * M + r) * Jp;
        const float* il = d.invlam + ((size_t)i * N + n) * Jp;
        float a = 0.f;
        for (int j = l + threadIdx.x; j < J; j += blockDim.x) {
            const float w = il[j - l];
            a += -logf(w) + abs2(yr[j]) * w;
        }
        acc += (double)a;
    }
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        d.cost_part[i] = t - 2.0 * (double)J * d.logdet[i];
    }
}

__global__ void cost_sum_kernel(const Shape s, const State d)
{
    __shared__ double part[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < s.F; i += blockDim.x) acc += d.cost_part[i];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *d.cost_out = t;
    }
}

cudaError_t launch_cost(const Shape& s, const State& d, cudaStream_t st)
{
    cost_bin_kernel<<<s.F, 256, 0, st>>>(s, d);
    cost_sum_kernel<<<1, 256, 0, st>>>(s, d);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ source images (Eqs. 23-24)
// Per bin: H = W_i^{-1} by Gauss-Jordan elimination with partial pivoting in FP64, then
// c_n[m][i][j] = sum_{l < L_n} H[m][(n,l)] y_{(n,l)}(j)  (projection-back form of the MWF).
__global__ void separate_kernel(const Shape s, const State d, float2* __restrict__ out)
{
    __shared__ double a[CTFMNMF_MAX_M][2 * CTFMNMF_MAX_M][2];   // [W | I] augmented, complex
    __shared__ float2 H[CTFMNMF_MAX_M][CTFMNMF_MAX_M];
    const int i = blockIdx.x;
    const int M = s.M, F = s.F, J = s.J, Jp = s.Jp;
    if (threadIdx.x == 0) {
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < 2 * M; ++q) {
                if (q < M) {
                    const float2 w = d.W[((size_t)i * M + p) * M + q];
                    a[p][q][0] = w.x;
                    a[p][q][1] = w.y;
                } else {
                    a[p][q][0] = (q - M == p) ? 1.0 : 0.0;
                    a[p][q][1] = 0.0;
                }
            }
        for (int c = 0; c < M; ++c) {
            int piv = c;
            double best = -1.0;
            for (int p = c; p < M; ++p) {
                const double m2 = a[p][c][0] * a[p][c][0] + a[p][c][1] * a[p][c][1];
                if (m2 > best) { best = m2; piv = p; }
            }
            if (piv != c)
                for (int q = 0; q < 2 * M; ++q)
                    for (int t = 0; t < 2; ++t) { double x = a[c][q][t]; a[c][q][t] = a[piv][q][t]; a[piv][q][t] = x; }
            // scale row c by 1/pivot
            const double pr = a[c][c][0], pi = a[c][c][1];
            const double den = pr * pr + pi * pi;
            const double ir = pr / den, ii = -pi / den;
            for (int q = 0; q < 2 * M; ++q) {
                const double xr = a[c][q][0], xi = a[c][q][1];
                a[c][q][0] = xr * ir - xi * ii;
                a[c][q][1] = xr * ii + xi * ir;
            }
            for (int p = 0; p < M; ++p) {
                if (p == c) continue;
                const double fr = a[p][c][0], fi = a[p][c][1];
                for (int q = 0; q < 2 * M; ++q) {
                    const double xr = a[c][q][0], xi = a[c][q][1];
                    a[p][q][0] -= fr * xr - fi * xi;
                    a[p][q][1] -= fr * xi + fi * xr;
                }
            }
        }
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < M; ++q) H[p][q] = make_float2((float)a[p][M + q][0], (float)a[p][M + q][1]);
    }
    __syncthreads();
    const float2* Yb = d.Y + (size_t)i * M * Jp;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        float2 yv[CTFMNMF_MAX_M];
        for (int r = 0; r < M; ++r) yv[r] = Yb[(size_t)r * Jp + j];
        for (int n = 0; n < s.N; ++n) {
            const int r0 = s.row0[n], Lp = s.Ln[n];
            for (int m = 0; m < M; ++m) {
                float2 c = make_float2(0.f, 0.f);
                for (int l = 0; l < Lp; ++l) {
                    const float2 h = H[m][r0 + l], v = yv[r0 + l];
                    c.x += h.x * v.x - h.y * v.y;
                    c.y += h.x * v.y + h.y * v.x;
                }
                out[(((size_t)n * M + m) * F + i) * J + j] = c;
            }
        }
    }
}

cudaError_t launch_separate(const Shape& s, const State& d, float2* out, cudaStream_t st)
{
    separate_kernel<<<s.F, 256, 0, st>>>(s, d, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ read-outs
__global__ void get_demixed_kernel(const Shape s, const State d, float2* __restrict__ out)
{
    const int i = blockIdx.x, r = blockIdx.y;
    const float2* src = d.Y + ((size_t)i * s.M + r) * s.Jp;
    float2* dst = out + ((size_t)r * s.F + i) * s.J;
    for (int j = threadIdx.x; j < s.J; j += blockDim.x) dst[j] = src[j];
}

cudaError_t launch_get_demixed(const Shape& s, const State& d, float2* out, cudaStream_t st)
{
    get_demixed_kernel<<<dim3(s.F, s.M), 256, 0, st>>>(s, d, out);
    return cudaGetLastError();
}

__global__ void get_nmf_kernel(const Shape s, const State d, float* __restrict__ T, float* __restrict__ V)
{
    const int N = s.N, F = s.F, B = s.B, J = s.J, Jp = s.Jp;
    const size_t nT = T ? (size_t)N * F * B : 0, nV = V ? (size_t)N * B * J : 0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nT + nV;
         e += (size_t)gridDim.x * blockDim.x) {
        if (e < nT) {
            const int k = (int)(e % B);
            const int i = (int)((e / B) % F);
            const int n = (int)(e / ((size_t)B * F));
            T[e] = d.T[(size_t)n * s.FBp + (size_t)i * B + k];
        } else {
            const size_t f = e - nT;
            const int j = (int)(f % J);
            V[f] = d.V[(f / J) * Jp + j];
        }
    }
}

cudaError_t launch_get_nmf(const Shape& s, const State& d, float* T, float* V, cudaStream_t st)
{
    get_nmf_kernel<<<256, 256, 0, st>>>(s, d, T, V);
    return cudaGetLastError();
}

}  // namespace ctf
