// Internal definitions shared by the CUDA translation units of libctfmnmf.
//
// Device data layout (one mixture, all resident in HBM):
//   Y      [F][M][Jp]  complex64  demixed extended rows, bin-major: one bin is one
//                                 contiguous block of M*Jp*8 bytes (Jp = J rounded up to 8)
//   X      [F][M][Jp]  complex64  the loaded observation in the same layout (IP update only)
//   W      [F][M][M]   complex64  row r of W_i holds w_r^H
//   logdet [F]         float64    log|det W_i|, tracked by the determinant lemma
//   T      [N][FBp]    float32    bases, T[n][i][k] at n*FBp + i*B + k (the API shape [N][F][B]
//                                 with each source block padded to 16 bytes)
//   V      [N][B][Jp]  float32    activations (padding frames are 0)
//   invlam [F][N][Jp]  float32    1/lambda_{n,i,j} for the current V and the bases T' before
//                                 the pending normalisation (padding 0): the bin phase
//                                 multiplies it by mu_{(n,0)}^2 = 1/scale_{(n,0)}^2
//   P      [F][N][Jp]  float32    delayed row power feeding the activation update
//   mupart [F][M]      float64    per-bin row power sums feeding the normalisation
//   scale  [M]         float32    pending normalisation 1/mu_r not yet applied to Y, W, T
//                                 and 1/lambda
//   ldm, lde [F]       f64, i32   running product of |det| factors (mantissa, exponent),
//                                 folded into logdet at the end of every iterate call
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ctfmnmf.h"

namespace ctf {

constexpr float kFloorNmf = 1e-12f;   // default floor of T and V after each multiplicative update
constexpr float kFloorPsd = 1e-18f;   // floor of lambda where it is formed

struct Shape {
    int M, N, B, F, J, Jp;
    int FBp;                    // per-source stride of T: F*B rounded up to a multiple of 4
    int Ln[CTFMNMF_MAX_M];
    int row_n[CTFMNMF_MAX_M];   // extended row r -> source n
    int row_l[CTFMNMF_MAX_M];   // extended row r -> tap l
    int row0[CTFMNMF_MAX_M];    // source n -> its tap-0 row
    int det_reduce;             // 1: every reduction in a fixed order (ctfmnmf_options)
    float floor_nmf;            // floor of T and V after each multiplicative update
                                // (ctfmnmf_options.eps_floor, default kFloorNmf)
    double invJ;                // 1/J in FP64 (the 1/J of Eq. 8 in the ISS normaliser)
};

struct State {
    float2* Y;
    float2* W;
    double* logdet;
    float* T;
    float* V;
    float* invlam;
    float* P;
    double* mupart;
    float* scale;
    float* detb;        // [F] the bin phase's |det W_i| factor of this iteration (pending scale
                        //     included), folded into ldm/lde by the frame phase
    double* ldm;        // [F] mantissa of the log-det product not yet folded into logdet
    int* lde;           // [F] its binary exponent
    unsigned* sync;     // grid barrier words: [0] abort, [1] arrivals, [2] generation
    int* flag;          // [0]: non-finite input seen, [1]: device wait timed out,
                        // [2]: NaN/Inf found after an iteration, [3]: a debug bounds check failed
    double* cost_part;  // [F] per-bin cost
    double* cost_out;   // [1]
    float2* staging;    // host-loaded STFT staging [M][F][J]
    float2* X;          // [F][M][Jp] observation kept for the IP update (null for ISS)
};

// Launchers (host functions; each enqueues its kernels on `st` and returns the
// cudaGetLastError() of the launch).
cudaError_t launch_load(const Shape& s, const State& d, const float2* X, cudaStream_t st);
cudaError_t launch_init_nmf(const Shape& s, const State& d, const float* T0, const float* V0,
                            uint64_t seed, cudaStream_t st);
cudaError_t launch_psd(const Shape& s, const State& d, cudaStream_t st);
cudaError_t launch_probe_fill(const Shape& s, const State& d, cudaStream_t st);
cudaError_t configure_bin_phase(const Shape& s);
cudaError_t launch_bin_phase(const Shape& s, const State& d, int v_tap0, cudaStream_t st);
// The bin phase with an explicit (frames per thread, threads) from bin_phase_candidates.
int bin_phase_candidates(int M, int J, int* fpts, int* nts);
cudaError_t configure_bin_phase_as(const Shape& s, int fpt, int nt);
cudaError_t launch_bin_phase_as(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st);
// IP update (Eqs. 9-10) in place of the ISS sweep, M <= 4 (bin_phase.cu)
cudaError_t configure_ip_bin_phase(const Shape& s);
cudaError_t launch_ip_bin_phase(const Shape& s, const State& d, int v_tap0, cudaStream_t st);
cudaError_t configure_frame_phase();
cudaError_t launch_frame_phase(const Shape& s, const State& d, int v_tap0, int normalize,
                               cudaStream_t st);
cudaError_t launch_finalize(const Shape& s, const State& d, cudaStream_t st);
// NaN/Inf scan of Y, T, V: sets flag[2] if any value is not finite (kernels.cu)
cudaError_t launch_finite_scan(const Shape& s, const State& d, cudaStream_t st);
cudaError_t launch_cost(const Shape& s, const State& d, cudaStream_t st);
cudaError_t launch_separate(const Shape& s, const State& d, float2* out, cudaStream_t st);
cudaError_t launch_get_demixed(const Shape& s, const State& d, float2* out, cudaStream_t st);
cudaError_t launch_get_nmf(const Shape& s, const State& d, float* T, float* V, cudaStream_t st);

// Persistent path: all iterations in one cooperative launch (persistent.cu).
struct PersistPlan {
    int ok;          // shape supported by the persistent kernel
    int fpt, gt;     // frames per thread, threads per group
    int groups;      // groups per CTA
    int gsm;         // shared floats per group
    int res_floats;  // shared floats per group for the resident rows and W_i (0: streaming)
    int fc;          // bins per frame-phase chunk
    int resident;    // 1: Y and W stay in shared memory across iterations
    int ctas;        // CTAs launched
    size_t smem;     // dynamic shared bytes per CTA
};
PersistPlan plan_persistent(const Shape& s);
cudaError_t launch_persistent(const Shape& s, const State& d, const PersistPlan& p, int n_iter,
                              int v_tap0, int normalize, unsigned long long timeout_ns, int skip_cta,
                              cudaStream_t st);

// Batched path (batch.cu): one descriptor per mixture, launch classes of equal template
// arguments; `work` lists the (mixture, bin) or (mixture, item) pair of every block.
struct MixDesc {
    Shape s;
    State d;
};
struct BatchClass {
    int M, fpt, nt, blocks;
    int N;             // contiguous-frame class (fpt == kBinContig): sources of every mixture;
                       // its bases-group count is kept in kb
    int kb;            // bases per basis-MU pass (4, 8, 10, 16), covering every B of the class
    size_t smem;
    int2* work;        // device [blocks]
};
cudaError_t launch_batch_bin(const BatchClass& c, const MixDesc* mixes, int v_tap0, cudaStream_t st,
                             bool configure);
int bases_class(int B);   // 4, 8, 10 or 16: the basis-MU pass width for B bases (bin_phase.cu)
cudaError_t configure_batch_frame();
int batch_frame_class(int B);
int batch_frame_chunk(int B, int BB);
cudaError_t launch_batch_frame(int BB, int exact, const MixDesc* mixes, const int2* work, int blocks, int v_tap0,
                               int normalize, cudaStream_t st);

// Long-J bin phase (cluster_bin.cu): one bin over a cluster of cl blocks of nt threads,
// jc frames each; used when the bin's frames do not fit one block.
struct ClusterPlan {
    int ok, cl, jc, nt;
};
ClusterPlan plan_cluster(const Shape& s);
cudaError_t configure_cluster_bin_phase(const Shape& s, const ClusterPlan& p);
cudaError_t launch_cluster_bin_phase(const Shape& s, const State& d, int v_tap0, const ClusterPlan& p,
                                     cudaStream_t st);
// Frames of one bin a cluster of 8 blocks can hold (host rule, before any device query).
inline int cluster_max_frames(int M) { return 8 * 512 * (M == 2 ? 8 : 4); }

// Contiguous-frame bin phase (bin_contig.cuh; bin_fpt code kBinContig): 8 consecutive frames
// per thread, compile-time default taps, M <= 4, J <= 4096.
constexpr int kBinContig = -8;
// Groups of 4 bases it is compiled for: 1 (B <= 4), 3 (B <= 12), 4 (B <= 16), 8 (B <= 32).
__host__ __device__ constexpr int contig_groups(int B) { return B <= 4 ? 1 : B <= 12 ? 3 : B <= 16 ? 4 : 8; }
bool contig_supported(const Shape& s);
int contig_threads(const Shape& s);
size_t contig_smem_bytes(const Shape& s, int nt);
// M, N and bases groups GB of the launch; mixes == nullptr: the two-kernel kernel over s, d (s.F blocks), else the
// batched kernel over `blocks` work items; cfg: raise the kernel's shared-memory limit only.
cudaError_t contig_dispatch(int M, int N, int GB, const Shape& s, const State& d, const MixDesc* mixes,
                            const int2* work, int blocks, int nt, size_t smem, int v_tap0, cudaStream_t st, bool cfg);

// Set the message that ctfmnmf_last_error(NULL) returns on this thread.
void set_thread_error(const char* msg);

// Frames per thread / threads per block chosen for the bin phase; false if unsupported.
bool bin_phase_config(int M, int J, int* fpt, int* threads);
size_t bin_phase_smem(const Shape& s);
// Shared floats of the bin phase for shape s with nt threads per block.
int bin_smem_floats(const Shape& s, int nt);

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {   // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float abs2(float2 a) { return a.x * a.x + a.y * a.y; }

// 1/x for normal positive x: the hardware reciprocal estimate refined by one Newton-Raphson
// step r <- r (2 - x r), which squares its relative error (about 1 ulp after the step).
__device__ __forceinline__ float recip(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r * fmaf(-x, r, 2.0f);
}

// Asynchronous global -> shared copies (cp.async): every thread issues its copies, then
// cp_async_wait() and a barrier make them visible. The 16-byte form reads through L2 only.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The ISS normaliser of Eq. 16 for p = r: 1 - z_r = q^{-1/2}, q = (1/J) sum_j phi_r |y_r|^2,
// formed and inverted in FP64 from the FP32 frame sum (invJ = 1/J in FP64); 1 for a row
// without energy. FP64 on this GPU issues at about 1/64 of the FP32 rate whatever the active
// lanes, so callers take the value off their critical path (it is needed only once the
// sweep is over, see bin_body).
__device__ __forceinline__ float iss_normaliser(float sum, double invJ)
{
    if (!(sum > 0.f)) return 1.0f;
    return (float)rsqrt((double)sum * invJ);
}

// The pending normalisation of Eqs. 19-21 applied to a stored 1/lambda (formed from the bases
// before it): 1/lambda'' = mu^2 / lambda' with mu = 1/s0, kept below the 1/floor of lambda.
__device__ __forceinline__ float scaled_invlam(float w, float fac)
{
    return fminf(w * fac, 1.0f / kFloorPsd);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace ctf
