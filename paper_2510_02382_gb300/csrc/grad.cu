// Backward pass of unrolled CTF-MNMF-ISS: hand-written adjoint of one iteration (Sec. III)
// and of the projection-back images (Eq. 24). Notation and buffers: grad.cuh.
//
// Per iteration t, in stream order:
//   A grad_norm_kernel     (bin, mixture)          e_r = sum Re(conj(gY') Y') + Re(conj(gW') W')
//                                                  + [l(r) = 0] 2 sum gT' T'   (the sigma sums);
//                                                  only for the first iteration reversed: kernel C
//                                                  forms the sums of the iteration before its own
//   B grad_vmu_kernel      (32 frames, source, mixture)  denV by a sweep over all bins; from
//                                                  dL/dV' the gradients of numV, denV and the
//                                                  direct part V' = V R of dL/dV
//   E grad_act_kernel      (256 frames x 32 bins, source, mixture)  the activation MU's
//                                                  per-bin adjoint parts (dL/dlambda', dL/dS,
//                                                  per-tile sums of dL/dT1 and the basis-MU
//                                                  denominator)
//   C grad_bin_kernel      (bin, mixture)          recompute the ISS sweep; adjoint of the
//                                                  normalisation, the basis MU (with kernel E's
//                                                  activation-MU parts) and the ISS sweep;
//                                                  writes dL/dY, dL/dW, dL/dT of the bin and the
//                                                  per-(bin, frame) terms kernel D needs
//   D grad_vgather_kernel  (128 frames x 32 bins, source, mixture)  dL/dV += sum over those
//                                                  bins of those terms (float atomics)
#include <stdio.h>

#include "grad_bin.cuh"

namespace ctf {
// ---------------------------------------------------------------- A: normalisation sums
template <int M>
__global__ void __launch_bounds__(256) grad_norm_kernel(const Shape s, const StatePtrs* __restrict__ nxt_tab,
                                                        const GradBufs g)
{
    __shared__ float red[8 * M];
    __shared__ float out[M];
    const int i = blockIdx.x, sm = blockIdx.y;
    const int N = s.N, B = s.B, F = s.F, J = s.J, Jp = s.Jp, FBp = s.FBp;
    const StatePtrs nxt = nxt_tab[sm];
    const float2* gYb = g.gY + ((size_t)sm * F + i) * M * Jp;
    const float2* Yb = nxt.Y + (size_t)i * M * Jp;
    float a[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
        a[r] = 0.f;
        for (int j = threadIdx.x; j < J; j += blockDim.x) {
            const float2 gy = gYb[(size_t)r * Jp + j], y = Yb[(size_t)r * Jp + j];
            a[r] = fmaf(gy.x, y.x, fmaf(gy.y, y.y, a[r]));
        }
    }
    if ((int)threadIdx.x < M * M) {
        const int p = threadIdx.x / M, c = threadIdx.x - p * M;
        const float2 gw = g.gW[(((size_t)sm * F + i) * M + p) * M + c];
        const float2 w = nxt.W[((size_t)i * M + p) * M + c];
#pragma unroll
        for (int r = 0; r < M; ++r)
            if (r == p) a[r] = fmaf(gw.x, w.x, fmaf(gw.y, w.y, a[r]));
    }
    for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
        const int n = t / B, k = t - n * B;
        const size_t o = (size_t)n * FBp + (size_t)i * B + k;
        const float v = 2.f * g.gT[(size_t)sm * N * FBp + o] * nxt.T[o];
#pragma unroll
        for (int r = 0; r < M; ++r)
            if (r == s.row0[n]) a[r] += v;
    }
    block_sum<M>(a, red, out);
    if ((int)threadIdx.x < M) atomicAdd(&g.e[sm * M + threadIdx.x], (double)out[threadIdx.x]);
}

// ---------------------------------------------------------------- B: activation-MU gradients
// Block = kVT frames x kVG bin groups: warp w sums the bins i = w mod kVG for its lane's frame,
// then the groups' partial denominators are added in shared memory and each warp finishes
// the bases k = w mod kVG.
constexpr int kVT = 32;    // frames per block (one per lane)
constexpr int kVG = 8;     // bin groups per block (one per warp)
constexpr int kIC = 256;   // bins staged per pass

template <int BB>
__global__ void __launch_bounds__(kVT * kVG) grad_vmu_kernel(const Shape s, const StatePtrs* __restrict__ cur_tab,
                                                             const StatePtrs* __restrict__ nxt_tab, const GradBufs g,
                                                             const int gin)
{
    constexpr int kSh = kIC * BB > kVG * BB * kVT ? kIC * BB : kVG * BB * kVT;
    __shared__ float sh[kSh];                          // T1 of kIC bins, then the partial denominators
    const int sm = blockIdx.z, n = blockIdx.y;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int j = blockIdx.x * kVT + lane;
    const int N = s.N, B = s.B, F = s.F, J = s.J, Jp = s.Jp, FBp = s.FBp;
    const StatePtrs cur = cur_tab[sm], nxt = nxt_tab[sm];
    const float s0 = g.sig[sm * s.M + s.row0[n]];
    const float inv = 1.f / (s0 * s0);                 // T1 = T' / sigma_{(n,0)}^2
    const bool live = j < J;
    float v[BB], den[BB];
#pragma unroll
    for (int k = 0; k < BB; ++k) {
        v[k] = (live && k < B) ? cur.V[((size_t)n * B + k) * Jp + j] : 0.f;
        den[k] = 0.f;
    }
    const float c = live ? (float)min(s.Ln[n], J - j) : 0.f;   // taps l with j + l < J
    for (int i0 = 0; i0 < F; i0 += kIC) {
        const int ic = min(kIC, F - i0);
        __syncthreads();
        for (int e = threadIdx.x; e < ic * BB; e += blockDim.x) {
            const int ii = e / BB, k = e - ii * BB;
            sh[e] = k < B ? nxt.T[(size_t)n * FBp + (size_t)(i0 + ii) * B + k] * inv : 0.f;
        }
        __syncthreads();
        if (live) {
            for (int ii = grp; ii < ic; ii += kVG) {
                const float* t1 = sh + ii * BB;
                float lam = 0.f;
#pragma unroll
                for (int k = 0; k < BB; ++k) lam = fmaf(t1[k], v[k], lam);
                const float w = c / fmaxf(lam, kFloorPsd);
#pragma unroll
                for (int k = 0; k < BB; ++k) den[k] = fmaf(t1[k], w, den[k]);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BB; ++k) sh[(grp * BB + k) * kVT + lane] = den[k];
    __syncthreads();
    if (j >= Jp) return;
    const size_t base = ((size_t)sm * N + n) * B * (size_t)Jp + j;
    for (int k = grp; k < B; k += kVG) {
        float dk = 0.f;
#pragma unroll
        for (int q = 0; q < kVG; ++q) dk += sh[(q * BB + k) * kVT + lane];
        const size_t idx = base + (size_t)k * Jp;
        float gn = 0.f, gd = 0.f, gv = 0.f;
        if (live) {
            const float g1 = g.gV[gin][idx];
            const float V1 = nxt.V[((size_t)n * B + k) * Jp + j], V = cur.V[((size_t)n * B + k) * Jp + j];
            if (V1 > s.floor_nmf && V > 0.f && dk > 0.f) {
                // V1 = V R, R = sqrt(numV / denV): dR/dnum = 1/(2 R den), dR/dden = -R/(2 den)
                const float R = V1 / V, gR = g1 * V;
                gn = gR / (2.f * R * dk);
                gd = -gR * R / (2.f * dk);
                gv = g1 * R;
            }
        }
        g.gnum[idx] = gn;
        g.gden[idx] = gd;
        g.gV[1 - gin][idx] = gv;
    }
}

// ---------------------------------------------------------------- E: activation-MU adjoint, per-bin parts
// For every (bin i, frame j) of one (source n, mixture): with T1 = T'/sigma_{(n,0)}^2, the
// delayed power S of |Y1|^2 = |Y'|^2 / sigma^2 over the source's taps, c the tap count and
// lambda' = T1 V: A = S / lambda'^2, dL/dlambda' = -2 A gA / lambda' - c gC / lambda'^2
// (0 where lambda' is floored) with gA = sum_k dL/dnumV T1, gC = sum_k dL/ddenV T1, and
// dL/dS = gA / lambda'^2, and 1/lambda of the iteration (lambda = T V, floored; 0 past J) for the
// per-bin kernel; per bin the sums over frames of dL/dT1 (sum_j dL/dnumV A +
// dL/ddenV c/lambda' + dL/dlambda' V) and of the basis-MU denominator (sum_j V c/lambda with
// lambda = T V). Block = kEW warps x 32 frames (one frame per lane) over kEI bins; V and the
// two gradient planes of its frames are staged once in shared memory for all of its bins.
// The per-bin sums go out per 32-frame tile (actp), added up by grad_bin_kernel.
// REG (B <= 8): each lane keeps its frame's V and gradient-plane values in registers across
// the bins, so a bin costs only the broadcast loads of its bases.
constexpr int kEW = 8;     // warps (32-frame tiles) per block
constexpr int kEI = 32;    // bins per block

template <bool REG>
__global__ void __launch_bounds__(kEW * 32, REG ? 4 : 1)
grad_act_kernel(const Shape s, const StatePtrs* __restrict__ cur_tab, const StatePtrs* __restrict__ nxt_tab,
                const GradBufs g)
{
    extern __shared__ float esm[];
    constexpr int FT = kEW * 32;                       // frames per block
    const int N = s.N, B = s.B, F = s.F, J = s.J, Jp = s.Jp, FBp = s.FBp, M = s.M;
    const int TB = REG ? 8 : B;                        // stride of the staged bases (REG: zero-padded to 8)
    const int sm = blockIdx.z / N, n = blockIdx.z - sm * N;
    const int j0 = blockIdx.x * FT, i0 = blockIdx.y * kEI;
    const int ic = min(kEI, F - i0);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    float* Vt = esm;                                   // [B][FT]
    float* Gn = Vt + B * FT;                           // [B][FT]
    float* Gd = Gn + B * FT;                           // [B][FT]
    float* T1s = Gd + B * FT;                          // [kEI][TB]
    float* Ts = T1s + kEI * TB;                        // [kEI][TB]
    const StatePtrs cur = cur_tab[sm], nxt = nxt_tab[sm];
    const float* sig = g.sig + sm * M;
    const int r0 = s.row0[n], Lq = s.Ln[n];
    const float s0 = sig[r0];
    const float inv = 1.f / (s0 * s0);
    const size_t pl = ((size_t)sm * N + n) * B * (size_t)Jp;     // [S][N][B][Jp] planes
    for (int e = tid; e < B * FT; e += blockDim.x) {
        const int k = e / FT, jj = e - k * FT, j = j0 + jj;
        float v = 0.f, gn = 0.f, gd = 0.f;
        if (j < J) {
            const size_t o = (size_t)k * Jp + j;
            v = cur.V[(size_t)n * B * Jp + o];
            gn = g.gnum[pl + o];
            gd = g.gden[pl + o];
        }
        Vt[e] = v;
        Gn[e] = gn;
        Gd[e] = gd;
    }
    for (int e = tid; e < ic * TB; e += blockDim.x) {
        const int ii = e / TB, k = e - ii * TB;
        const size_t o = (size_t)n * FBp + (size_t)(i0 + ii) * B + k;
        T1s[e] = k < B ? nxt.T[o] * inv : 0.f;
        Ts[e] = k < B ? cur.T[o] : 0.f;
    }
    __syncthreads();
    if (j0 + w * 32 >= Jp) return;                     // a warp past the last frame tile
    const int jj = w * 32 + lane, j = j0 + jj;
    const bool live = j < J;
    const float c = live ? (float)min(Lq, J - j) : 0.f;
    float isg[kGradMaxM];                              // 1 / sigma^2 of the source's rows
#pragma unroll
    for (int l = 0; l < kGradMaxM; ++l) {
        const float sg = l < Lq ? sig[r0 + l] : 0.f;
        isg[l] = sg > 0.f ? 1.f / (sg * sg) : 0.f;
    }
    const int tiles = (Jp + 31) >> 5, tile = (j0 >> 5) + w;
    // per-bin pointers, advanced bin by bin: the rows (n, 0..) at this frame, the two output
    // planes at this frame, the tile's partial sums
    const float2* Yr = nxt.Y + ((size_t)i0 * M + r0) * Jp + (live ? j : 0);
    const size_t ystep = (size_t)M * Jp;
    const size_t q0 = (((size_t)sm * N + n) * F + i0) * (size_t)Jp + j;
    float* part = g.actp + ((((size_t)sm * N + n) * tiles + tile) * F + i0) * (size_t)(2 * B);
    float vr[8], gnr[8], gdr[8];                       // REG: this frame's V, dL/dnumV, dL/ddenV
    if constexpr (REG) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            vr[k] = k < B ? Vt[k * FT + jj] : 0.f;
            gnr[k] = k < B ? Gn[k * FT + jj] : 0.f;
            gdr[k] = k < B ? Gd[k * FT + jj] : 0.f;
        }
    }
    for (int ii = 0; ii < ic; ++ii, Yr += ystep, part += 2 * B) {
        float A = 0.f, cc = 0.f, gp = 0.f, gs = 0.f, ci = 0.f, ilam = 0.f;
        if (live) {
            float S = 0.f;
#pragma unroll
            for (int l = 0; l < kGradMaxM; ++l)
                if (l < Lq && j + l < J) S = fmaf(abs2(Yr[(size_t)l * (Jp + 1)]), isg[l], S);
            float raw = 0.f, gA = 0.f, gC = 0.f, lam = 0.f;
            if constexpr (REG) {
                const float4* t1 = reinterpret_cast<const float4*>(T1s + ii * 8);
                const float4* t = reinterpret_cast<const float4*>(Ts + ii * 8);
                const float4 a1 = t1[0], b1 = t1[1], a0 = t[0], b0 = t[1];
                const float tk1[8] = {a1.x, a1.y, a1.z, a1.w, b1.x, b1.y, b1.z, b1.w};
                const float tk[8] = {a0.x, a0.y, a0.z, a0.w, b0.x, b0.y, b0.z, b0.w};
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    raw = fmaf(tk1[k], vr[k], raw);
                    lam = fmaf(tk[k], vr[k], lam);
                    gA = fmaf(gnr[k], tk1[k], gA);
                    gC = fmaf(gdr[k], tk1[k], gC);
                }
            } else {
                const float* t1 = T1s + ii * TB;
                const float* t = Ts + ii * TB;
#pragma unroll 4
                for (int k = 0; k < B; ++k) {
                    const float v = Vt[k * FT + jj];
                    raw = fmaf(t1[k], v, raw);
                    lam = fmaf(t[k], v, lam);
                    gA = fmaf(Gn[k * FT + jj], t1[k], gA);
                    gC = fmaf(Gd[k * FT + jj], t1[k], gC);
                }
            }
            const float il = __frcp_rn(fmaxf(raw, kFloorPsd));
            A = S * il * il;
            cc = c * il;
            gp = raw > kFloorPsd ? (-2.f * A * il * gA - cc * il * gC) : 0.f;
            gs = gA * il * il;
            ilam = __frcp_rn(fmaxf(lam, kFloorPsd));
            ci = c * ilam;
        }
        if (j < Jp) {
            const size_t q = q0 + (size_t)ii * Jp;
            g.glp[q] = gp;
            g.gsa[q] = gs;
            g.ilp[q] = ilam;
        }
        for (int kb = 0; kb < B; kb += 8) {
            float a[16];
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int k = kb + kk;
                if constexpr (REG) {
                    a[kk] = fmaf(gnr[kk], A, fmaf(gdr[kk], cc, gp * vr[kk]));
                    a[8 + kk] = vr[kk] * ci;
                } else {
                    const float v = k < B ? Vt[k * FT + jj] : 0.f;
                    a[kk] = k < B ? fmaf(Gn[k * FT + jj], A, fmaf(Gd[k * FT + jj], cc, gp * v)) : 0.f;
                    a[8 + kk] = v * ci;
                }
            }
            reduce_scatter<16>(a, lane);
            if (!(lane & 1)) {
                const int v = lane >> 1, k = kb + (v & 7);
                if (k < B) part[v < 8 ? k : B + k] = a[0];
            }
        }
    }
}

inline size_t act_smem(const Shape& s)
{
    const int tb = s.B <= 8 ? 8 : s.B;                 // the staged bases' stride (see TB)
    return sizeof(float) * ((size_t)s.B * 3 * kEW * 32 + (size_t)2 * kEI * tb);
}

// ---------------------------------------------------------------- D: gather dL/dV over bins
constexpr int kID = 32;    // bins per block (blocks of one frame tile add into dL/dV)

template <int BB>
__global__ void __launch_bounds__(kGradTile) grad_vgather_kernel(const Shape s, const StatePtrs* __restrict__ cur_tab,
                                                                 const StatePtrs* __restrict__ nxt_tab,
                                                                 const GradBufs g, const int gout)
{
    __shared__ float T1s[kID * BB], Ts[kID * BB], gns[kID * BB], gds[kID * BB];
    const int N = s.N, B = s.B, F = s.F, J = s.J, Jp = s.Jp, FBp = s.FBp;
    const int tiles = (Jp + kGradTile - 1) / kGradTile;
    const int sm = blockIdx.z, n = blockIdx.y, j = (blockIdx.x % tiles) * kGradTile + threadIdx.x;
    const StatePtrs cur = cur_tab[sm], nxt = nxt_tab[sm];
    const float s0 = g.sig[sm * s.M + s.row0[n]];
    const float inv = 1.f / (s0 * s0);
    const bool live = j < J;
    const size_t tb = (size_t)sm * N * FBp + (size_t)n * FBp;
    const size_t rows = ((size_t)sm * N + n) * F;
    float v[BB], acc[BB];
#pragma unroll
    for (int k = 0; k < BB; ++k) {
        v[k] = (live && k < B) ? cur.V[((size_t)n * B + k) * Jp + j] : 0.f;
        acc[k] = 0.f;
    }
    const float c = live ? (float)min(s.Ln[n], J - j) : 0.f;
    {
        const int i0 = blockIdx.x / tiles * kID;          // this block's bins [i0, i0 + ic)
        const int ic = min(kID, F - i0);
        for (int e = threadIdx.x; e < ic * BB; e += blockDim.x) {
            const int ii = e / BB, k = e - ii * BB;
            const size_t o = (size_t)(i0 + ii) * B + k;
            const bool ok = k < B;
            T1s[e] = ok ? nxt.T[(size_t)n * FBp + o] * inv : 0.f;
            Ts[e] = ok ? cur.T[(size_t)n * FBp + o] : 0.f;
            gns[e] = ok ? g.gnT[tb + o] : 0.f;
            gds[e] = ok ? g.gdT[tb + o] : 0.f;
        }
        __syncthreads();
        if (live) {
#pragma unroll 4
            for (int ii = 0; ii < ic; ++ii) {
                const size_t q = (rows + i0 + ii) * (size_t)Jp + j;
                const float glp = g.glp[q], glt = g.glt[q], A = g.aq[q];
                const float* t = Ts + ii * BB;
                float lam = 0.f;
#pragma unroll
                for (int k = 0; k < BB; ++k) lam = fmaf(t[k], v[k], lam);
                const float ci = c / fmaxf(lam, kFloorPsd);
                const float* t1 = T1s + ii * BB;
                const float* gn = gns + ii * BB;
                const float* gd = gds + ii * BB;
#pragma unroll
                for (int k = 0; k < BB; ++k)
                    acc[k] = fmaf(glp, t1[k], fmaf(glt, t[k], fmaf(gn[k], A, fmaf(gd[k], ci, acc[k]))));
            }
        }
    }
    if (!live) return;
    const size_t base = ((size_t)sm * N + n) * B * (size_t)Jp + j;
#pragma unroll
    for (int k = 0; k < BB; ++k)
        if (k < B) atomicAdd(&g.gV[gout][base + (size_t)k * Jp], acc[k]);
}

// ---------------------------------------------------------------- images (Eq. 24) adjoint
// c_n = sum_{r in n} H[:, r] y_r with H = W^{-1}: dL/dy_r = H[:, r]^H dL/dc_{n(r)},
// dL/dH = sum_j dL/dc y^H, dL/dW = -H^H (dL/dH) H^H.
template <int M>
__global__ void __launch_bounds__(256) grad_head_kernel(const Shape s, const StatePtrs* __restrict__ live_tab,
                                                        const float2* __restrict__ gC, const GradBufs g)
{
    constexpr int V = 2 * M * M;
    __shared__ double a[M][2 * M][2];
    __shared__ float2 H[M][M];
    __shared__ float red[8 * V];
    __shared__ float out[V];
    const int i = blockIdx.x, sm = blockIdx.y;
    const int N = s.N, B = s.B, F = s.F, J = s.J, Jp = s.Jp, FBp = s.FBp;
    const StatePtrs lv = live_tab[sm];
    if (threadIdx.x == 0) {
        // Gauss-Jordan elimination with partial pivoting on [W | I] in FP64
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < 2 * M; ++q) {
                if (q < M) {
                    const float2 w = lv.W[((size_t)i * M + p) * M + q];
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
                if (m2 > best) {
                    best = m2;
                    piv = p;
                }
            }
            if (piv != c)
                for (int q = 0; q < 2 * M; ++q)
                    for (int t = 0; t < 2; ++t) {
                        const double x = a[c][q][t];
                        a[c][q][t] = a[piv][q][t];
                        a[piv][q][t] = x;
                    }
            const double pr = a[c][c][0], pi = a[c][c][1], den = pr * pr + pi * pi;
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
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    const float2* Yb = lv.Y + (size_t)i * M * Jp;
    float2* gYo = g.gY + ((size_t)sm * F + i) * M * Jp;
    for (int j = threadIdx.x; j < Jp; j += blockDim.x) {
        float2 gyv[M];
#pragma unroll
        for (int r = 0; r < M; ++r) gyv[r] = make_float2(0.f, 0.f);
        if (j < J) {
#pragma unroll
            for (int r = 0; r < M; ++r) {
                const float2 yr = Yb[(size_t)r * Jp + j];
                const int n = s.row_n[r];
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const float2 gc = gC[((((size_t)sm * N + n) * M + m) * F + i) * J + j];
                    const float2 u = cmulf(conjf2(H[m][r]), gc);
                    gyv[r] = make_float2(gyv[r].x + u.x, gyv[r].y + u.y);
                    const float2 w = cmul_conj(gc, yr);
                    acc[2 * (m * M + r)] += w.x;
                    acc[2 * (m * M + r) + 1] += w.y;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < M; ++r) gYo[(size_t)r * Jp + j] = gyv[r];
    }
    block_sum<V>(acc, red, out);
    if (threadIdx.x == 0) {
        float2 gH[M][M], P[M][M];
        for (int m = 0; m < M; ++m)
            for (int r = 0; r < M; ++r) gH[m][r] = make_float2(out[2 * (m * M + r)], out[2 * (m * M + r) + 1]);
        for (int m = 0; m < M; ++m)          // P = gH H^H
            for (int c = 0; c < M; ++c) {
                float2 t = make_float2(0.f, 0.f);
                for (int r = 0; r < M; ++r) {
                    const float2 u = cmul_conj(gH[m][r], H[c][r]);
                    t = make_float2(t.x + u.x, t.y + u.y);
                }
                P[m][c] = t;
            }
        for (int p = 0; p < M; ++p)          // dL/dW = -H^H P
            for (int c = 0; c < M; ++c) {
                float2 t = make_float2(0.f, 0.f);
                for (int m = 0; m < M; ++m) {
                    const float2 u = cmulf(conjf2(H[m][p]), P[m][c]);
                    t = make_float2(t.x + u.x, t.y + u.y);
                }
                g.gW[(((size_t)sm * F + i) * M + p) * M + c] = make_float2(-t.x, -t.y);
            }
    }
    for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
        const int n = t / B, k = t - n * B;
        g.gT[(size_t)sm * N * FBp + (size_t)n * FBp + (size_t)i * B + k] = 0.f;
    }
}

// ---------------------------------------------------------------- inputs
// Y_0 = X (W_0 = I): dL/dX[m][i][j] = dL/dY_0[i][m][j]; T, V were floored on entry, so the
// gradient passes where the stored initial value is above the floor.
__global__ void grad_inputs_kernel(const Shape s, const StatePtrs* __restrict__ init_tab, const GradBufs g,
                                   float2* __restrict__ gX, float* __restrict__ gT0)
{
    const int i = blockIdx.x, m = blockIdx.y, sm = blockIdx.z;
    const int M = s.M, N = s.N, B = s.B, F = s.F, J = s.J, Jp = s.Jp, FBp = s.FBp;
    const float2* src = g.gY + (((size_t)sm * F + i) * M + m) * Jp;
    float2* dst = gX + (((size_t)sm * M + m) * F + i) * J;
    for (int j = threadIdx.x; j < J; j += blockDim.x) dst[j] = src[j];
    if (m == 0) {
        const StatePtrs in = init_tab[sm];
        for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
            const int n = t / B, k = t - n * B;
            const size_t o = (size_t)n * FBp + (size_t)i * B + k;
            gT0[(((size_t)sm * N + n) * F + i) * B + k] = in.T[o] > s.floor_nmf ? g.gT[(size_t)sm * N * FBp + o] : 0.f;
        }
    }
}

__global__ void grad_v0_kernel(const Shape s, const StatePtrs* __restrict__ init_tab, const float* __restrict__ gV,
                               float* __restrict__ gV0)
{
    const int row = blockIdx.x, sm = blockIdx.y;     // row = n * B + k
    const int N = s.N, B = s.B, J = s.J, Jp = s.Jp;
    const float* vin = init_tab[sm].V + (size_t)row * Jp;
    const float* src = gV + ((size_t)sm * N * B + row) * Jp;
    float* dst = gV0 + ((size_t)sm * N * B + row) * J;
    for (int j = threadIdx.x; j < J; j += blockDim.x) dst[j] = vin[j] > s.floor_nmf ? src[j] : 0.f;
}

// ---------------------------------------------------------------- state copies (checkpoints)
__global__ void grad_copy_kernel(const Shape s, const StatePtrs* __restrict__ src_tab,
                                 const StatePtrs* __restrict__ dst_tab)
{
    const int sm = blockIdx.y;
    const StatePtrs a = src_tab[sm], b = dst_tab[sm];
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nY = (size_t)s.F * s.M * s.Jp / 2;            // float4 = two complex values
    const size_t nW = (size_t)s.F * s.M * s.M;
    const size_t nT = (size_t)s.N * s.FBp / 4;
    const size_t nV = (size_t)s.N * s.B * s.Jp / 4;
    for (size_t e = t0; e < nY; e += stride) reinterpret_cast<float4*>(b.Y)[e] = reinterpret_cast<const float4*>(a.Y)[e];
    for (size_t e = t0; e < nW; e += stride) b.W[e] = a.W[e];
    for (size_t e = t0; e < nT; e += stride) reinterpret_cast<float4*>(b.T)[e] = reinterpret_cast<const float4*>(a.T)[e];
    for (size_t e = t0; e < nV; e += stride) reinterpret_cast<float4*>(b.V)[e] = reinterpret_cast<const float4*>(a.V)[e];
}

// ---------------------------------------------------------------- finalize with sigma record
// As finalize_kernel (the pending normalisation applied to Y, W, log|det|, T, 1/lambda) for every
// mixture of the batch; also records sigma_r = the applied scale. One block per (bin, mixture)
// covering all of its rows with 16-byte accesses (two complex values, four 1/lambda). With a
// snapshot table (snap != NULL) the normalised Y, W, T and a copy of V go to snap[mixture]
// instead (the state at the start of the next iteration, kept for the backward pass) and the
// live state keeps its pending normalisation, which the next bin phase applies as it loads.
__global__ void grad_finalize_kernel(const MixDesc* __restrict__ mixes, float* __restrict__ sig,
                                     const StatePtrs* __restrict__ snap)
{
    const int i = blockIdx.x, sm = blockIdx.y;
    const Shape& s = mixes[sm].s;
    const State& d = mixes[sm].d;
    const int M = s.M, N = s.N, B = s.B, Jp = s.Jp;
    if (i >= s.F) return;
    __shared__ float sc[CTFMNMF_MAX_M];
    if ((int)threadIdx.x < M) sc[threadIdx.x] = d.scale[threadIdx.x];
    __syncthreads();
    const StatePtrs sp = snap ? snap[sm] : StatePtrs{nullptr, nullptr, nullptr, nullptr};
    const int R4 = Jp >> 1;                              // float4 per row of Y
    float4* Yb = reinterpret_cast<float4*>(d.Y + (size_t)i * M * Jp);
    float4* Ys = snap ? reinterpret_cast<float4*>(sp.Y + (size_t)i * M * Jp) : nullptr;
    for (int e = threadIdx.x; e < M * R4; e += blockDim.x) {
        const float c = sc[e / R4];
        const float4 v = Yb[e];
        const float4 o = make_float4(v.x * c, v.y * c, v.z * c, v.w * c);
        if (Ys) Ys[e] = o;
        else Yb[e] = o;
    }
    if ((int)threadIdx.x < M * M) {
        float2* w = d.W + (size_t)i * M * M + threadIdx.x;
        const float c = sc[threadIdx.x / M];
        const float2 o = make_float2(w->x * c, w->y * c);
        if (snap) sp.W[(size_t)i * M * M + threadIdx.x] = o;
        else *w = o;
    }
    if (snap) {
        for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
            const int n = t / B, k = t - n * B;
            const float c = sc[s.row0[n]];
            const size_t o = (size_t)n * s.FBp + (size_t)i * B + k;
            sp.T[o] = d.T[o] * (c * c);
        }
        const size_t nV4 = (size_t)N * B * Jp / 4;     // V [N][B][Jp], split over the bins
        for (size_t e = (size_t)i * blockDim.x + threadIdx.x; e < nV4; e += (size_t)s.F * blockDim.x)
            reinterpret_cast<float4*>(sp.V)[e] = reinterpret_cast<const float4*>(d.V)[e];
        if (i == 0 && (int)threadIdx.x < M) sig[sm * M + threadIdx.x] = sc[threadIdx.x];
        return;
    }
    if (threadIdx.x == 0) {
        double f = d.ldm[i];
        for (int p = 0; p < M; ++p) f *= (double)sc[p];
        d.logdet[i] += log(f) + (double)d.lde[i] * 0.69314718055994530942;
        d.ldm[i] = 1.0;
        d.lde[i] = 0;
    }
    for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
        const int n = t / B, k = t - n * B;
        const float c = sc[s.row0[n]];
        d.T[(size_t)n * s.FBp + (size_t)i * B + k] *= c * c;
    }
    const int L4 = Jp >> 2;                              // float4 per row of 1/lambda
    float4* il = reinterpret_cast<float4*>(d.invlam + (size_t)i * N * Jp);
    for (int e = threadIdx.x; e < N * L4; e += blockDim.x) {
        const float c = sc[s.row0[e / L4]];
        const float fac = 1.0f / (c * c);
        const float4 v = il[e];
        il[e] = make_float4(scaled_invlam(v.x, fac), scaled_invlam(v.y, fac), scaled_invlam(v.z, fac),
                            scaled_invlam(v.w, fac));
    }
    if (i == 0 && (int)threadIdx.x < M) sig[sm * M + threadIdx.x] = sc[threadIdx.x];
}

__global__ void grad_reset_scale_kernel(const MixDesc* __restrict__ mixes)
{
    const MixDesc& md = mixes[blockIdx.x];
    if ((int)threadIdx.x < md.s.M) md.d.scale[threadIdx.x] = 1.f;
}

// ---------------------------------------------------------------- MSE loss head
__global__ void __launch_bounds__(256) grad_mse_kernel(const size_t count, const float2* __restrict__ C,
                                                       const float2* __restrict__ R, double* __restrict__ loss,
                                                       const double* __restrict__ dloss, float2* __restrict__ gC)
{
    __shared__ double part[8];
    const double inv = 1.0 / (double)count;
    const float gs = gC ? (float)(2.0 * (dloss ? *dloss : 1.0) * inv) : 0.f;
    double acc = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const float2 c = C[e], r = R[e];
        const float2 d = make_float2(c.x - r.x, c.y - r.y);
        acc += (double)(d.x * d.x + d.y * d.y);
        if (gC) gC[e] = make_float2(gs * d.x, gs * d.y);
    }
    if (!loss) return;
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(loss, t * inv);
    }
}

// ---------------------------------------------------------------- host launchers
// kernel C instantiations in grad_bin_m<M>.cu
cudaError_t grad_bin_m2(const Shape& s, int S, const StatePtrs* cur, const StatePtrs* nxt, const GradBufs& g,
                        cudaStream_t st, bool configure);
cudaError_t grad_bin_m3(const Shape& s, int S, const StatePtrs* cur, const StatePtrs* nxt, const GradBufs& g,
                        cudaStream_t st, bool configure);
cudaError_t grad_bin_m4(const Shape& s, int S, const StatePtrs* cur, const StatePtrs* nxt, const GradBufs& g,
                        cudaStream_t st, bool configure);

namespace {

int pick_bb(int B) { return B <= 4 ? 4 : B <= 8 ? 8 : B <= 16 ? 16 : 32; }

cudaError_t launch_bin(const Shape& s, int S, const StatePtrs* cur, const StatePtrs* nxt, const GradBufs& g,
                       cudaStream_t st, bool configure)
{
    switch (s.M) {
        case 2: return grad_bin_m2(s, S, cur, nxt, g, st, configure);
        case 3: return grad_bin_m3(s, S, cur, nxt, g, st, configure);
        case 4: return grad_bin_m4(s, S, cur, nxt, g, st, configure);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t grad_configure(const Shape& s)
{
    GradBufs g;
    memset(&g, 0, sizeof(g));
    const cudaError_t e = s.B <= 8 ? cudaFuncSetAttribute(grad_act_kernel<true>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)act_smem(s))
                                   : cudaFuncSetAttribute(grad_act_kernel<false>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)act_smem(s));
    if (e != cudaSuccess) return e;
    return launch_bin(s, 1, nullptr, nullptr, g, nullptr, true);
}

size_t grad_act_partials(const Shape& s, int S)
{
    return (size_t)S * s.N * (size_t)((s.Jp + 31) / 32) * s.F * 2 * s.B;
}

cudaError_t grad_enqueue_iteration(const Shape& s, int S, const StatePtrs* cur, const StatePtrs* nxt,
                                   const GradBufs& g, int gin, bool first, cudaStream_t st, int* kernels)
{
    *kernels = 4;
    if (first) {
        cudaError_t e = cudaMemsetAsync(g.e, 0, sizeof(double) * S * s.M, st);
        if (e != cudaSuccess) return e;
        switch (s.M) {
            case 2: grad_norm_kernel<2><<<dim3(s.F, S), 256, 0, st>>>(s, nxt, g); break;
            case 3: grad_norm_kernel<3><<<dim3(s.F, S), 256, 0, st>>>(s, nxt, g); break;
            case 4: grad_norm_kernel<4><<<dim3(s.F, S), 256, 0, st>>>(s, nxt, g); break;
            default: return cudaErrorInvalidValue;
        }
        *kernels = 5;
    }
    cudaError_t e = cudaMemsetAsync(g.e_prev, 0, sizeof(double) * S * s.M, st);
    if (e != cudaSuccess) return e;
    const dim3 vgrid((s.Jp + kVT - 1) / kVT, s.N, S);
    switch (pick_bb(s.B)) {
        case 4: grad_vmu_kernel<4><<<vgrid, kVT * kVG, 0, st>>>(s, cur, nxt, g, gin); break;
        case 8: grad_vmu_kernel<8><<<vgrid, kVT * kVG, 0, st>>>(s, cur, nxt, g, gin); break;
        case 16: grad_vmu_kernel<16><<<vgrid, kVT * kVG, 0, st>>>(s, cur, nxt, g, gin); break;
        default: grad_vmu_kernel<32><<<vgrid, kVT * kVG, 0, st>>>(s, cur, nxt, g, gin); break;
    }
    const dim3 egrid((s.Jp + kEW * 32 - 1) / (kEW * 32), (s.F + kEI - 1) / kEI, s.N * S);
    if (s.B <= 8) grad_act_kernel<true><<<egrid, kEW * 32, act_smem(s), st>>>(s, cur, nxt, g);
    else grad_act_kernel<false><<<egrid, kEW * 32, act_smem(s), st>>>(s, cur, nxt, g);
    const dim3 fgrid((s.Jp + kGradTile - 1) / kGradTile, s.N, S);
    e = launch_bin(s, S, cur, nxt, g, st, false);
    if (e != cudaSuccess) return e;
    const dim3 dgrid(fgrid.x * ((s.F + kID - 1) / kID), s.N, S);
    switch (pick_bb(s.B)) {
        case 4: grad_vgather_kernel<4><<<dgrid, kGradTile, 0, st>>>(s, cur, nxt, g, 1 - gin); break;
        case 8: grad_vgather_kernel<8><<<dgrid, kGradTile, 0, st>>>(s, cur, nxt, g, 1 - gin); break;
        case 16: grad_vgather_kernel<16><<<dgrid, kGradTile, 0, st>>>(s, cur, nxt, g, 1 - gin); break;
        default: grad_vgather_kernel<32><<<dgrid, kGradTile, 0, st>>>(s, cur, nxt, g, 1 - gin); break;
    }
    return cudaGetLastError();
}

cudaError_t grad_launch_head(const Shape& s, int S, const StatePtrs* live, const float2* gC, const GradBufs& g,
                             cudaStream_t st)
{
    switch (s.M) {
        case 2: grad_head_kernel<2><<<dim3(s.F, S), 256, 0, st>>>(s, live, gC, g); break;
        case 3: grad_head_kernel<3><<<dim3(s.F, S), 256, 0, st>>>(s, live, gC, g); break;
        case 4: grad_head_kernel<4><<<dim3(s.F, S), 256, 0, st>>>(s, live, gC, g); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t grad_launch_inputs(const Shape& s, int S, const StatePtrs* init, const GradBufs& g, int gcur,
                               float2* gX, float* gT0, float* gV0, cudaStream_t st)
{
    grad_inputs_kernel<<<dim3(s.F, s.M, S), 256, 0, st>>>(s, init, g, gX, gT0);
    grad_v0_kernel<<<dim3(s.N * s.B, S), 256, 0, st>>>(s, init, g.gV[gcur], gV0);
    return cudaGetLastError();
}

cudaError_t grad_launch_copy(const Shape& s, int S, const StatePtrs* src, const StatePtrs* dst, cudaStream_t st)
{
    grad_copy_kernel<<<dim3(64, S), 256, 0, st>>>(s, src, dst);
    return cudaGetLastError();
}

cudaError_t grad_launch_finalize(const Shape& s, int S, const MixDesc* mixes, float* sig, cudaStream_t st,
                                 const StatePtrs* snap)
{
    grad_finalize_kernel<<<dim3(s.F, S), 256, 0, st>>>(mixes, sig, snap);
    if (!snap) grad_reset_scale_kernel<<<S, 32, 0, st>>>(mixes);   // with a snapshot the scale stays pending
    return cudaGetLastError();
}

cudaError_t grad_launch_mse(size_t count, const float2* C, const float2* Cref, double* loss, const double* dloss,
                            float2* gC, cudaStream_t st)
{
    if (loss) {
        const cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), st);
        if (e != cudaSuccess) return e;
    }
    grad_mse_kernel<<<1024, 256, 0, st>>>(count, C, Cref, loss, dloss, gC);
    return cudaGetLastError();
}

}  // namespace ctf
