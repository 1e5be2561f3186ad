// Bin phase of the two-kernel path: one CTA per frequency bin runs the ISS sweep (or, for
// handles created with the IP update, the IP sweep of Eqs. 9-10) and the basis update of
// Sec. III for its bin (device code in phases.cuh, kernels in bin_phase_kernels.cuh). This
// file holds the configuration and the dispatch over M.
#include "bin_contig.cuh"

namespace ctf {

// contiguous-frame instantiations in bin_contig_m<M>.cu
cudaError_t contig_launch_m2(int N, int GB, const Shape& s, const State& d, const MixDesc* mixes, const int2* work,
                             int blocks, int nt, size_t smem, int v_tap0, cudaStream_t st, bool cfg);
cudaError_t contig_launch_m3(int N, int GB, const Shape& s, const State& d, const MixDesc* mixes, const int2* work,
                             int blocks, int nt, size_t smem, int v_tap0, cudaStream_t st, bool cfg);
cudaError_t contig_launch_m4(int N, int GB, const Shape& s, const State& d, const MixDesc* mixes, const int2* work,
                             int blocks, int nt, size_t smem, int v_tap0, cudaStream_t st, bool cfg);

bool contig_supported(const Shape& s)
{
    if (s.M < 2 || s.M > 4 || s.N < 1 || s.N > s.M) return false;
    for (int n = 0; n < s.N; ++n)
        if (s.Ln[n] != s.M / s.N + (n < s.M % s.N ? 1 : 0)) return false;
    return s.Jp % 8 == 0 && s.Jp <= kContigFpt * kContigMaxThreads;
}

int contig_threads(const Shape& s) { return (s.Jp / kContigFpt + 31) / 32 * 32; }

size_t contig_smem_bytes(const Shape& s, int nt)
{
    return sizeof(float) * (size_t)contig_smem_layout(s.M, s.N, s.B, s.Jp, nt).total;
}

cudaError_t contig_dispatch(int M, int N, int GB, const Shape& s, const State& d, const MixDesc* mixes,
                            const int2* work, int blocks, int nt, size_t smem, int v_tap0, cudaStream_t st, bool cfg)
{
    switch (M) {
        case 2: return contig_launch_m2(N, GB, s, d, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 3: return contig_launch_m3(N, GB, s, d, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
        case 4: return contig_launch_m4(N, GB, s, d, mixes, work, blocks, nt, smem, v_tap0, st, cfg);
    }
    return cudaErrorInvalidValue;
}

// instantiations in bin_phase_m<M>.cu
cudaError_t bin_phase_m2(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg);
cudaError_t bin_phase_m3(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg);
cudaError_t bin_phase_m4(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg);
cudaError_t bin_phase_m5(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg);
cudaError_t bin_phase_m6(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg);
cudaError_t bin_phase_m7(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg);
cudaError_t bin_phase_m8(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg);
cudaError_t ip_bin_phase_m2(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg);
cudaError_t ip_bin_phase_m3(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg);
cudaError_t ip_bin_phase_m4(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st, bool cfg);

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
    return sizeof(float) * (size_t)bin_smem_layout(s.M, s.N, s.Jp, nt).total;
}

// Every (frames per thread, threads) the bin phase can run this shape with: for each of
// 1, 2, 4 (up to 256 threads) and 8 (M <= 4, up to 512 threads) the threads that cover J.
int bin_phase_candidates(int M, int J, int* fpts, int* nts)
{
    static const int cands[4] = {1, 2, 4, 8};
    int k = 0;
    for (int c = 0; c < 4; ++c) {
        const int f = cands[c];
        if (M * f > 32) break;
        const int cap = f == 8 ? 512 : 256;
        const int nt = (J + f - 1) / f;
        if (nt > cap) continue;
        fpts[k] = f;
        nts[k] = nt < 64 ? 64 : ((nt + 31) / 32) * 32;
        ++k;
    }
    return k;
}

int bin_smem_floats(const Shape& s, int nt) { return bin_smem_layout(s.M, s.N, s.Jp, nt).total; }

int bases_class(int B) { return B <= 4 ? 4 : B <= 8 ? 8 : B <= 10 ? 10 : 16; }

static cudaError_t dispatch(const Shape& s, const State& d, int v_tap0, cudaStream_t st, bool cfg, int fpt = 0,
                            int nt = 0)
{
    if (fpt == kBinContig) {
        if (!contig_supported(s) || nt != contig_threads(s)) return cudaErrorInvalidValue;
        return contig_dispatch(s.M, s.N, contig_groups(s.B), s, d, nullptr, nullptr, s.F, nt, contig_smem_bytes(s, nt),
                               v_tap0, st, cfg);
    }
    if (fpt == 0 && !bin_phase_config(s.M, s.J, &fpt, &nt)) return cudaErrorInvalidValue;
    switch (s.M) {
        case 2: return bin_phase_m2(s, d, v_tap0, fpt, nt, st, cfg);
        case 3: return bin_phase_m3(s, d, v_tap0, fpt, nt, st, cfg);
        case 4: return bin_phase_m4(s, d, v_tap0, fpt, nt, st, cfg);
        case 5: return bin_phase_m5(s, d, v_tap0, fpt, nt, st, cfg);
        case 6: return bin_phase_m6(s, d, v_tap0, fpt, nt, st, cfg);
        case 7: return bin_phase_m7(s, d, v_tap0, fpt, nt, st, cfg);
        case 8: return bin_phase_m8(s, d, v_tap0, fpt, nt, st, cfg);
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

cudaError_t configure_bin_phase_as(const Shape& s, int fpt, int nt)
{
    State none = {};
    return dispatch(s, none, 0, nullptr, true, fpt, nt);
}

cudaError_t launch_bin_phase_as(const Shape& s, const State& d, int v_tap0, int fpt, int nt, cudaStream_t st)
{
    return dispatch(s, d, v_tap0, st, false, fpt, nt);
}

static cudaError_t dispatch_ip(const Shape& s, const State& d, int v_tap0, cudaStream_t st, bool cfg)
{
    int fpt = 0, nt = 0;
    if (!bin_phase_config(s.M, s.J, &fpt, &nt)) return cudaErrorInvalidValue;
    switch (s.M) {
        case 2: return ip_bin_phase_m2(s, d, v_tap0, fpt, nt, st, cfg);
        case 3: return ip_bin_phase_m3(s, d, v_tap0, fpt, nt, st, cfg);
        case 4: return ip_bin_phase_m4(s, d, v_tap0, fpt, nt, st, cfg);
    }
    return cudaErrorInvalidValue;
}

cudaError_t configure_ip_bin_phase(const Shape& s)
{
    State none = {};
    return dispatch_ip(s, none, 0, nullptr, true);
}

cudaError_t launch_ip_bin_phase(const Shape& s, const State& d, int v_tap0, cudaStream_t st)
{
    return dispatch_ip(s, d, v_tap0, st, false);
}

}  // namespace ctf
