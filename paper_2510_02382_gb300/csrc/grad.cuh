// Differentiable form (grad.cu, grad_api.cpp): buffers and launchers of the backward pass.
//
// Notation of one iteration t of a mixture (Sec. III), state S_t = (Y, W, T, V) at its start:
//   lambda = max(T V, floor)                       phi_r(j) = 1/lambda_{n(r), j - l(r)}
//   ISS sweep (Eqs. 11-16)          Y, W  -> Y1, W1
//   basis MU (Eq. 17)               T     -> T1 = max(T sqrt(numT / denT), floor)
//   activation MU (Eq. 18, all taps) V    -> V1 = max(V sqrt(numV / denV), floor), with T1
//   normalisation (Eqs. 19-21)      sigma_r = (sum |Y1_r|^2 / (F J))^{-1/2}
//                                   Y' = sigma Y1, W' = sigma W1, T'_n = sigma_{(n,0)}^2 T1_n, V' = V1
// The backward pass of iteration t reads S_t, S_{t+1} = (Y', W', T', V') and the recorded
// sigma_t, and turns the gradients with respect to S_{t+1} into those with respect to S_t.
#pragma once

#include "internal.cuh"

namespace ctf {

constexpr int kGradMaxM = 4;        // most extended rows of the differentiable form
constexpr int kGradMaxJ = 2048;     // most frames
constexpr int kGradTile = 128;      // frames per block of the frame-parallel kernels

// One mixture's iteration state (device pointers in the handle layout of internal.cuh).
struct StatePtrs {
    float2* Y;
    float2* W;
    float* T;
    float* V;
};

// Gradient buffers of a batch of S mixtures of one shape (device; [S] leading).
struct GradBufs {
    float2* gY;          // [S][F][M][Jp]  dL/dY (of the state the pass has reached)
    float2* gW;          // [S][F][M][M]   dL/dW
    float* gT;           // [S][N][FBp]    dL/dT
    float* gV[2];        // [S][N][B][Jp]  dL/dV, double-buffered: one read, one written
    float* gnum;         // [S][N][B][Jp]  dL/d numV (activation MU numerator)
    float* gden;         // [S][N][B][Jp]  dL/d denV
    float* glp;          // [S][N][F][Jp]  dL/d lambda' (lambda of T1 and V; 0 where floored)
    float* glt;          // [S][N][F][Jp]  dL/d lambda (of T and V; 0 where floored)
    float* aq;           // [S][N][F][Jp]  A = (delayed power) / lambda^2 of the basis MU
    float* gsa;          // [S][N][F][Jp]  dL/d(delayed power) through the activation MU
    float* ilp;          // [S][N][F][Jp]  1/lambda of the iteration's T and V (0 past J)
    float* actp;         // [S][N][ceil(Jp/32)][F][2B]  per 32-frame tile: sums of dL/dT1 and of
                         //                the basis-MU denominator over its frames
    float* gnT;          // [S][N][FBp]    dL/d numT (basis MU numerator)
    float* gdT;          // [S][N][FBp]    dL/d denT
    double* e;           // [S][M]         normalisation sums of the iteration being reversed
                         //                (grad_norm_kernel, or the previous reversed iteration)
    double* e_prev;      // [S][M]         the same sums of the iteration before it, accumulated by
                         //                the per-bin adjoint from its outputs (zeroed before it)
    const float* sig;    // [S][M]         sigma_r of the iteration being reversed
};

cudaError_t grad_configure(const Shape& s);
size_t grad_act_partials(const Shape& s, int S);   // floats of GradBufs::actp
// Enqueue the backward pass of one iteration (kernels A-E of grad.cu); gin selects the
// gV buffer that holds dL/dV'; the other receives dL/dV. first: the first iteration reversed,
// whose normalisation sums kernel A forms (later ones get them from the per-bin adjoint of the
// iteration reversed before, in g.e). Returns the kernels launched in *kernels.
cudaError_t grad_enqueue_iteration(const Shape& s, int S, const StatePtrs* cur, const StatePtrs* nxt,
                                   const GradBufs& g, int gin, bool first, cudaStream_t st, int* kernels);
cudaError_t grad_launch_head(const Shape& s, int S, const StatePtrs* live, const float2* gC, const GradBufs& g,
                             cudaStream_t st);
cudaError_t grad_launch_inputs(const Shape& s, int S, const StatePtrs* init, const GradBufs& g, int gcur,
                               float2* gX, float* gT0, float* gV0, cudaStream_t st);
cudaError_t grad_launch_copy(const Shape& s, int S, const StatePtrs* src, const StatePtrs* dst, cudaStream_t st);
// snap (device [S], or NULL): also write the normalised state there (the next iteration's start)
cudaError_t grad_launch_finalize(const Shape& s, int S, const MixDesc* mixes, float* sig, cudaStream_t st,
                                 const StatePtrs* snap = nullptr);
cudaError_t grad_launch_mse(size_t count, const float2* C, const float2* Cref, double* loss,
                            const double* dloss, float2* gC, cudaStream_t st);

}  // namespace ctf
