// The solver handle behind ctfmnmf_t (host side), shared by the C ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include "internal.cuh"

using ctf::Shape;
using ctf::State;

struct ctfmnmf {
    Shape s;
    State d;
    ctfmnmf_options opt;
    int L;
    int device;
    cudaStream_t stream;        // user stream (nullptr = legacy default stream)
    cudaStream_t capture;       // private stream used to capture the iteration graph
    bool loaded;
    cudaGraphExec_t graph;
    int graph_iters;
    double* host_cost;          // pinned one-double landing buffer
    float2* sepbuf;             // device images for ctfmnmf_get_separated_host (lazy)
    long long launches;         // kernels enqueued so far
    ctf::PersistPlan plan;      // persistent-path plan for this shape on this device
    ctf::ClusterPlan cplan;     // long-J bin phase (ok when one block cannot hold a bin)
    int bin_fpt, bin_nt;        // frames per thread and threads of the bin phase (0: default)
    int path;                   // CTFMNMF_PATH_TWO_KERNEL or CTFMNMF_PATH_PERSISTENT
    int skip_cta;               // test hook: block that skips its first barrier arrival
    unsigned long long timeout_ns;
    char err[256];
};

#include <nvtx3/nvToolsExt.h>

namespace ctf {
// An NVTX range over a host call (visible in Nsight timelines; costs nothing when no tool
// is attached).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// kernels enqueued by one ctfmnmf_iterate of n_iter iterations on the two-kernel path
long long iteration_kernels(int n_iter, bool scan);
// finalize kernels (pending normalisation) launched at the end of every iterate call
constexpr int kFinalizeKernels = 2;
}  // namespace ctf
