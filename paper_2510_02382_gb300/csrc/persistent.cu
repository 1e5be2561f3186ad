// Host side of the persistent path: planning (group size, shared memory, residency,
// grid size from the occupancy calculator) and the cooperative launch. The kernel is in
// persistent_kernel.cuh, instantiated per M in persistent_m*.cu.
#include <string.h>

#include "persistent_kernel.cuh"

namespace ctf {

// ----------------------------------------------------------------------------- planning
static const void* select_kernel(int M, int BB)
{
    switch (M) {
        case 2: return persistent_ptr_m2(BB);
        case 3: return persistent_ptr_m3(BB);
        case 4: return persistent_ptr_m4(BB);
        case 5: return persistent_ptr_m5(BB);
        case 6: return persistent_ptr_m6(BB);
        case 7: return persistent_ptr_m7(BB);
        case 8: return persistent_ptr_m8(BB);
    }
    return nullptr;
}

static int persist_bb(int B) { return B <= 4 ? 4 : B <= 8 ? 8 : B <= 10 ? 10 : B <= 16 ? 16 : 0; }

PersistPlan plan_persistent(const Shape& s)
{
    PersistPlan p;
    memset(&p, 0, sizeof(p));
    const int BB = persist_bb(s.B);
    if (BB == 0 || s.M < 2 || s.M > 8) return p;
    p.fpt = s.M <= 4 ? 8 : 4;
    int gt = (s.J + p.fpt - 1) / p.fpt;
    gt = ((gt + 31) / 32) * 32;
    if (gt < 64) gt = 64;
    if (gt > kPersistThreads) return p;
    p.gt = gt;
    int dev = 0, optin = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return p;
    const int static_bytes = 1024;                       // scales, scratch, barrier word
    const int bin_floats = bin_smem_layout(s.M, s.N, s.Jp, gt).total;
    const int res_floats = ((2 * s.M * s.Jp + 2 * s.M * s.M) + 3) & ~3;
    const void* k = select_kernel(s.M, BB);
    if (!k) return p;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
        cudaGetLastError();
        return p;
    }
    for (int resident = 1; resident >= 0; --resident) {
        for (int groups = kPersistThreads / gt; groups >= 1; --groups) {
            // the frame phase runs on the whole CTA over the groups' work regions
            const int nt = groups * gt;
            const int fixed = BB == 4 ? frame_smem_fixed<4>(nt) : BB == 8 ? frame_smem_fixed<8>(nt)
                            : BB == 10 ? frame_smem_fixed<10>(nt) : frame_smem_fixed<16>(nt);
            const int frame_min = fixed + 64 * (s.B + kFrameTile);
            int gsm = bin_floats;
            if (groups * gsm < frame_min) gsm = (frame_min + groups - 1) / groups;
            gsm = (gsm + 3) & ~3;
            const size_t smem = (size_t)groups * (gsm + (resident ? res_floats : 0)) * 4;
            if (smem + fa.sharedSizeBytes + static_bytes > (size_t)optin) continue;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, smem) != cudaSuccess || per_sm < 1) {
                cudaGetLastError();
                continue;
            }
            const int ctas = per_sm * sms;
            if (resident && (long long)ctas * groups < s.F) continue;
            p.groups = groups;
            p.gsm = gsm;
            p.res_floats = resident ? res_floats : 0;
            p.fc = frame_chunk(groups * gsm, s.B, fixed);
            p.resident = resident;
            p.ctas = ctas;
            p.smem = smem;
            p.ok = p.fc >= 4;
            return p;
        }
    }
    return p;
}

cudaError_t launch_persistent(const Shape& s, const State& d, const PersistPlan& p, int n_iter,
                              int v_tap0, int normalize, unsigned long long timeout_ns, int skip_cta,
                              cudaStream_t st)
{
    if (!p.ok) return cudaErrorInvalidValue;
    const void* k = select_kernel(s.M, persist_bb(s.B));
    if (!k || s.Jp % 8 != 0 || (p.fc * s.B) % 4 != 0) return cudaErrorInvalidValue;
    // reset the barrier words (epochs restart at 1 every launch; an aborted launch may have
    // left the abort word set)
    cudaError_t e = cudaMemsetAsync(d.sync, 0, 32 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    PersistArgs pa;
    pa.n_iter = n_iter;
    pa.gt = p.gt;
    pa.groups = p.groups;
    pa.gsm = p.gsm;
    pa.res_floats = p.res_floats;
    pa.fc = p.fc;
    pa.resident = p.resident;
    pa.v_tap0 = v_tap0;
    pa.normalize = normalize;
    pa.skip_cta = skip_cta;
    pa.timeout_ns = timeout_ns;
    Shape sc = s;
    State dc = d;
    void* args[] = {&sc, &dc, &pa};
    return cudaLaunchCooperativeKernel(k, dim3(p.ctas), dim3(p.groups * p.gt), args, p.smem, st);
}

}  // namespace ctf
