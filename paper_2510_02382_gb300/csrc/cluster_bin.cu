// Long-J bin phase: one bin split over a thread-block cluster of CL blocks (2..8), each
// holding a contiguous chunk of Jc frames of the bin's rows. Every sum over frames the bin
// phase needs (the ISS sums of Eq. 16 at each step, the row powers of Eq. 19, the basis-MU
// numerator and denominator of Eq. 17) is reduced inside each block and then across the
// cluster through distributed shared memory; the delayed power near a chunk's end reads the
// next block's |y|^2 the same way. Every block computes the same z from the same cluster
// totals, so W and the log-det factor agree across the cluster; block 0 stores them.
// Used when a bin's frames do not fit one block (bin_phase_config fails); the frame phase
// is unchanged.
#include <cooperative_groups.h>

#include "phases.cuh"

namespace cg = cooperative_groups;

namespace ctf {

constexpr int kClusterThreads = 512;

struct ClusterSmem {
    int sq, A, C, acc, total;    // float offsets: |y|^2 [M][Jc], A and C [N][Jc], MU sums [N*B][2]
};

__host__ __device__ inline ClusterSmem cluster_smem_layout(int M, int N, int B, int Jc)
{
    ClusterSmem L;
    L.sq = 0;
    L.A = L.sq + M * Jc;
    L.C = L.A + N * Jc;
    L.acc = L.C + N * Jc;
    L.total = L.acc + 2 * N * B + 8 * 2;           // + row powers [8] (and padding)
    L.total = (L.total + 3) & ~3;
    return L;
}

// Blocks per SM the register budget is sized for: two when a thread's rows are fewer than 16
// complex values (64 registers), so that one cluster's barrier waits overlap another's work.
template <int M, int FPT>
constexpr int cluster_min_blocks() { return M * FPT < 16 ? 2 : 1; }

template <int M, int FPT>
__global__ void __launch_bounds__(kClusterThreads, cluster_min_blocks<M, FPT>())
cluster_bin_kernel(const Shape s, const State d, const int v_tap0, const int Jc)
{
    constexpr int NV = 3 * M - 2;                   // d_p (M real), n_p for p != r (M-1 complex)
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks(), q = (int)cl.block_rank();
    const int i = blockIdx.x / CL;
    const int j0 = q * Jc;
    const int N = s.N, B = s.B, J = s.J, Jp = s.Jp;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
    extern __shared__ float4 csm4[];
    float* csm = reinterpret_cast<float*>(csm4);
    const ClusterSmem L = cluster_smem_layout(M, N, B, Jc);
    float* sq = csm + L.sq;
    float* Aw = csm + L.A;
    float* Cw = csm + L.C;
    float* acc = csm + L.acc;                       // [N*B][2] then row powers [M]
    float* rpw = acc + 2 * N * B;
    __shared__ float xb[2][32];                     // this block's ISS sums, double-buffered by step
    __shared__ float red[16][32];
    __shared__ float tot[32];
    __shared__ float s_scale[CTFMNMF_MAX_M];
    __shared__ float s_fac[CTFMNMF_MAX_M];          // per source: mu_{(n,0)}^2 for the stored 1/lambda

    if (tid < CTFMNMF_MAX_M) s_scale[tid] = tid < M ? d.scale[tid] : 1.f;
    if (tid < N) {
        const float s0 = d.scale[s.row0[tid]];
        s_fac[tid] = 1.0f / (s0 * s0);
    }
    for (int t = tid; t < 2 * N * B + M; t += NT) acc[t] = 0.f;
    __syncthreads();

    // ---- this block's frames of the bin's rows (pending scale applied), W columns, weights
    // delayed weights phi_r(j) = 1/lambda_{n(r),i,j-l(r)} (0 for j < l(r)): in registers when
    // they fit beside the rows, else read again (through L1) at each use
    constexpr bool kPhiReg = M * FPT <= 16;
    constexpr int PR = kPhiReg ? M : 1, PF = kPhiReg ? FPT : 1;
    float2 y[M][FPT];
    float phi[PR][PF];
    const float2* Yb = d.Y + (size_t)i * M * Jp;
    const float* il = d.invlam + (size_t)i * N * Jp;
#pragma unroll
    for (int r = 0; r < M; ++r) {
        const int n = s.row_n[r], l = s.row_l[r];
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int jl = tid + f * NT, j = j0 + jl;
            float2 v = make_float2(0.f, 0.f);
            if (jl < Jc && j < Jp) {
                v = __ldcg(Yb + (size_t)r * Jp + j);
                v = make_float2(v.x * s_scale[r], v.y * s_scale[r]);
            }
            y[r][f] = v;
            if (kPhiReg)
                phi[r % PR][f % PF] =
                    (jl < Jc && j < J && j >= l) ? scaled_invlam(__ldcg(il + (size_t)n * Jp + j - l), s_fac[n]) : 0.f;
        }
    }
    auto phi_at = [&](int p, int f) -> float {
        if (kPhiReg) return phi[p % PR][f % PF];
        const int jl = tid + f * NT, j = j0 + jl, l = s.row_l[p];
        const int n = s.row_n[p];
        return (jl < Jc && j < J && j >= l) ? scaled_invlam(__ldg(il + (size_t)n * Jp + j - l), s_fac[n]) : 0.f;
    };
    float2 wcol[M];                                 // threads < M: column tid of W_i
    if (tid < M) {
#pragma unroll
        for (int p = 0; p < M; ++p) {
            const float2 w = __ldcg(d.W + ((size_t)i * M + p) * M + tid);
            wcol[p] = make_float2(w.x * s_scale[p], w.y * s_scale[p]);
        }
    }

    // ---- ISS sweep (Eqs. 11-16) with cluster-wide sums; the normaliser of row r (FP64) is
    //      applied after the sweep, as in bin_body (every later step is homogeneous in row r)
    __shared__ float s_scr[CTFMNMF_MAX_M];
    float detf = 1.0f;
#pragma unroll
    for (int r = 0; r < M; ++r) {
        float a[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) a[k] = 0.f;
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const float2 yr = y[r][f];
            const float pr = abs2(yr);
#pragma unroll
            for (int p = 0; p < M; ++p) {
                const float ph = phi_at(p, f);
                a[p] = fmaf(ph, pr, a[p]);
                if (p != r) {
                    const int c = M + 2 * (p - (p > r ? 1 : 0));
                    const float2 cc = cmul_conj(y[p][f], yr);
                    a[c] = fmaf(ph, cc.x, a[c]);
                    a[c + 1] = fmaf(ph, cc.y, a[c + 1]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float v = warp_sum(a[k]);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (tid < NV) {
            float t = 0.f;
            for (int w = 0; w < NW; ++w) t += red[w][tid];
            xb[r & 1][tid] = t;
        }
        cl.sync();                                  // every block's sums of this step are in place
        if (tid < CL * NV) {                         // one remote read per thread, then a local sum
            const int b = tid / NV, v = tid - b * NV;
            red[b][v] = cl.map_shared_rank(&xb[r & 1][0], b)[v];
        }
        __syncthreads();
        if (tid < NV) {
            float t = 0.f;
            for (int b = 0; b < CL; ++b) t += red[b][tid];
            tot[tid] = t;
        }
        __syncthreads();
        float2 z[M];
#pragma unroll
        for (int p = 0; p < M; ++p) {
            z[p] = make_float2(0.f, 0.f);
            if (p != r && tot[p] > 0.f) {
                const int c = M + 2 * (p - (p > r ? 1 : 0));
                z[p] = make_float2(tot[c] / tot[p], tot[c + 1] / tot[p]);
            }
        }
        if (tid == 0) s_scr[r] = tot[r];            // the sum J q_r, inverted after the sweep
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
    if (warp == 0) {                                // FP64 normalisers, one row per lane of warp 0
        __syncwarp();
        const float sc = iss_normaliser(lane < M ? s_scr[lane] : 0.f, s.invJ);
        __syncwarp();
        if (lane < M) s_scr[lane] = sc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < M; ++r) {
        const float sc = s_scr[r];
        detf *= sc;
#pragma unroll
        for (int f = 0; f < FPT; ++f) y[r][f] = make_float2(y[r][f].x * sc, y[r][f].y * sc);
        if (tid < M) wcol[r] = make_float2(wcol[r].x * sc, wcol[r].y * sc);
    }

    // ---- rows out, |y|^2 for the delayed power, row-power partials
    float2* Yo = d.Y + (size_t)i * M * Jp;
    float rp[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
        rp[r] = 0.f;
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int jl = tid + f * NT, j = j0 + jl;
            if (jl < Jc) {
                const float p2 = abs2(y[r][f]);
                sq[r * Jc + jl] = p2;
                rp[r] += p2;
                if (j < Jp) __stcg(Yo + (size_t)r * Jp + j, y[r][f]);
            }
        }
        const float v = warp_sum(rp[r]);
        if (lane == 0) {                            // fixed order (below), or shared atomics
            if (s.det_reduce) red[warp][r] = v;
            else atomicAdd(&rpw[r], v);
        }
    }
    cl.sync();                                      // every block's |y|^2 is in place
    if (s.det_reduce && tid < M) {
        float t = 0.f;
        for (int w = 0; w < NW; ++w) t += red[w][tid];
        rpw[tid] = t;
    }

    // ---- delayed power P_n(j) = sum_{l < L_n, j + l < J} |y_{(n,l)}(j + l)|^2 (the next
    //      block's first frames past this chunk's end), basis-MU weights A = P / lambda^2 and
    //      C = (taps counted) / lambda
    const float* sq_next = q + 1 < CL ? cl.map_shared_rank(sq, q + 1) : sq;
    float* Pout = d.P + (size_t)i * N * Jp;
#pragma unroll 4
    for (int e = tid; e < N * Jc; e += NT) {
        const int n = e / Jc, jl = e - n * Jc, j = j0 + jl;
        const float w = j < J ? scaled_invlam(__ldcg(il + (size_t)n * Jp + j), s_fac[n]) : 0.f;   // 1/lambda_{n,i,j}
        const int r0 = s.row0[n], lq = min(s.Ln[n], J - j);            // taps l with j + l < J
        float P = 0.f;
        for (int l = 0; l < lq; ++l) {
            const int jj = jl + l;
            P += jj < Jc ? sq[(r0 + l) * Jc + jj] : sq_next[(r0 + l) * Jc + jj - Jc];
        }
        const float cnt = lq > 0 ? (float)lq : 0.f;
        Aw[n * Jc + jl] = P * w * w;
        Cw[n * Jc + jl] = cnt * w;
        if (j < Jp) __stcg(Pout + (size_t)n * Jp + j, v_tap0 ? (j < J ? sq[r0 * Jc + jl] : 0.f) : P);
    }
    __syncthreads();

    // ---- basis MU sums over this block's frames, per (source, base)
    const int jend = max(0, min(Jc, J - j0));       // this block's valid frames
    for (int t = warp; t < N * B; t += NW) {
        const int n = t / B, k = t - n * B;
        const float* Vr = d.V + ((size_t)n * B + k) * Jp + j0;
        const float* An = Aw + n * Jc;
        const float* Cn = Cw + n * Jc;
        float num = 0.f, den = 0.f;
#pragma unroll 8
        for (int jl = lane; jl < jend; jl += 32) {   // independent loads: let them overlap
            const float v = __ldcg(Vr + jl);
            num = fmaf(v, An[jl], num);
            den = fmaf(v, Cn[jl], den);
        }
        num = warp_sum(num);
        den = warp_sum(den);
        if (lane == 0) {
            acc[2 * t] = num;
            acc[2 * t + 1] = den;
        }
    }
    cl.sync();                                      // every block's MU sums and row powers are in place

    if (q == 0) {
        for (int t = tid; t < N * B; t += NT) {
            float num = 0.f, den = 0.f;
            for (int b = 0; b < CL; ++b) {
                const float* pa = cl.map_shared_rank(acc, b);
                num += pa[2 * t];
                den += pa[2 * t + 1];
            }
            const int n = t / B, k = t - n * B;
            const float s0 = s_scale[s.row0[n]];
            float* Tp = d.T + (size_t)n * s.FBp + (size_t)i * B + k;
            const float tcur = __ldcg(Tp) * (s0 * s0);
            const float tn = (den > 0.f) ? tcur * sqrtf(num / den) : tcur;
            __stcg(Tp, fmaxf(tn, s.floor_nmf));
        }
        if (tid < M) {
            double t = 0.0;                         // the bin's row power in FP64 (Eq. 19)
            for (int b = 0; b < CL; ++b) t += (double)cl.map_shared_rank(rpw, b)[tid];
            __stcg(d.mupart + (size_t)i * M + tid, t);
#pragma unroll
            for (int p = 0; p < M; ++p) __stcg(d.W + ((size_t)i * M + p) * M + tid, wcol[p]);
        }
        if (tid == 0) d.detb[i] = det_factor<M>(detf, s_scale);   // folded by the frame phase
    }
    cl.sync();                                      // no block leaves while its shared memory is read
}

// ---------------------------------------------------------------- host side
namespace {

int cluster_fpt(int M) { return M == 2 ? 8 : 4; }

template <int M, int FPT>
cudaError_t launch_cl(const Shape& s, const State& d, int v_tap0, const ClusterPlan& p, cudaStream_t st, bool cfg)
{
    const size_t smem = sizeof(float) * (size_t)cluster_smem_layout(M, s.N, s.B, p.jc).total;
    if (cfg) return cudaFuncSetAttribute(cluster_bin_kernel<M, FPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3(s.F * p.cl);
    c.blockDim = dim3(p.nt);
    c.dynamicSmemBytes = smem;
    c.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    c.attrs = attr;
    c.numAttrs = 1;
    return cudaLaunchKernelEx(&c, cluster_bin_kernel<M, FPT>, s, d, v_tap0, p.jc);
}

cudaError_t dispatch_cl(const Shape& s, const State& d, int v_tap0, const ClusterPlan& p, cudaStream_t st, bool cfg)
{
    switch (s.M) {
        case 2: return launch_cl<2, 8>(s, d, v_tap0, p, st, cfg);
        case 3: return launch_cl<3, 4>(s, d, v_tap0, p, st, cfg);
        case 4: return launch_cl<4, 4>(s, d, v_tap0, p, st, cfg);
        case 5: return launch_cl<5, 4>(s, d, v_tap0, p, st, cfg);
        case 6: return launch_cl<6, 4>(s, d, v_tap0, p, st, cfg);
        case 7: return launch_cl<7, 4>(s, d, v_tap0, p, st, cfg);
        case 8: return launch_cl<8, 4>(s, d, v_tap0, p, st, cfg);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

// The smallest cluster (2, 4 or 8 blocks) whose chunks fit one block: Jc = the bin's frames
// over CL, rounded up to 8, at most 512 threads x FPT frames, and the shared memory fitting
// the device's opt-in limit.
ClusterPlan plan_cluster(const Shape& s)
{
    ClusterPlan p = {0, 0, 0, 0};
    if (s.M < 2 || s.M > CTFMNMF_MAX_M) return p;
    const int fpt = cluster_fpt(s.M);
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return p;
    }
    for (int cl = 2; cl <= 8; cl *= 2) {
        const int jc = ((s.Jp + cl - 1) / cl + 7) / 8 * 8;
        int nt = ((jc + fpt - 1) / fpt + 31) / 32 * 32;
        if (nt < 64) nt = 64;
        if (nt > kClusterThreads) continue;
        const size_t smem = sizeof(float) * (size_t)cluster_smem_layout(s.M, s.N, s.B, jc).total;
        if (smem + 8192 > (size_t)optin) continue;
        p.ok = 1;
        p.cl = cl;
        p.jc = jc;
        p.nt = nt;
        return p;
    }
    return p;
}

cudaError_t configure_cluster_bin_phase(const Shape& s, const ClusterPlan& p)
{
    State none = {};
    return dispatch_cl(s, none, 0, p, nullptr, true);
}

cudaError_t launch_cluster_bin_phase(const Shape& s, const State& d, int v_tap0, const ClusterPlan& p,
                                     cudaStream_t st)
{
    return dispatch_cl(s, d, v_tap0, p, st, false);
}

}  // namespace ctf
