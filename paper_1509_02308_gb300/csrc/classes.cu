// S7 support: the miss-rate table of a plan and the answer classes of the
// candidates under it.
//
// The learned inverse reads a trace of mean latencies t = t0 + t_m r over the
// 512 plan points (Sec. 4.1), r being each point's miss rate after warm-up.
// pchase_miss_rates turns the simulator's per-item counts into that table;
// pchase_answer_classes groups candidates whose rates lie within a tolerance of
// each other at every point (single linkage), since no observation of mean
// latencies separates them, and names each group by its lowest index.
#include "pchase_internal.cuh"

namespace pchase {
namespace {

// rates[g * P + p] = counts[(g * P + p) * 2 + 1] / measured[p], divided in
// double and rounded once to float.
__global__ void miss_rates_kernel(const uint64_t *counts, uint32_t G, uint32_t P,
                                  const uint64_t *measured, float *rates) {
    const uint64_t n = (uint64_t)G * P;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t m = measured[i % P];
        rates[i] = m ? (float)((double)counts[2 * i + 1] / (double)m) : 0.0f;
    }
}

// Block i compares row i with every row j > i, one warp per row j at a time:
// the lanes walk the points 32 at a time (coalesced) and the pair is close
// when every |r_i - r_j| (exact in double) is <= tol.  Close pairs set both
// adjacency bits.
__global__ void __launch_bounds__(256) adjacency_kernel(const float *rates, uint32_t G, uint32_t P,
                                                        double tol, uint32_t *adj,
                                                        uint32_t words) {
    const uint32_t i = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *ri = rates + (uint64_t)i * P;
    for (uint32_t j = i + 1 + warp; j < G; j += blockDim.x >> 5) {
        const float *rj = rates + (uint64_t)j * P;
        bool close = true;
        for (uint32_t p0 = 0; p0 < P && close; p0 += 32) {
            const uint32_t p = p0 + lane;
            const bool ok = p >= P || fabs((double)ri[p] - (double)rj[p]) <= tol;
            close = __all_sync(kFull, ok);
        }
        if (close && lane == 0) {
            atomicOr(&adj[(uint64_t)i * words + (j >> 5)], 1u << (j & 31));
            atomicOr(&adj[(uint64_t)j * words + (i >> 5)], 1u << (i & 31));
        }
    }
}

// One block: label[i] starts at i and drops to the smallest label among i's
// neighbours until nothing changes, which leaves every row labelled with the
// lowest index of its connected component.  A component's diameter bounds
// the rounds; G rounds always suffice.
__global__ void __launch_bounds__(1024) components_kernel(const uint32_t *adj, uint32_t G,
                                                          uint32_t words, uint32_t *label) {
    __shared__ int changed;
    for (uint32_t i = threadIdx.x; i < G; i += blockDim.x) label[i] = i;
    for (uint32_t round = 0; round <= G; ++round) {
        __syncthreads();
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < G; i += blockDim.x) {
            uint32_t best = label[i];
            const uint32_t *row = adj + (uint64_t)i * words;
            for (uint32_t w = 0; w < words; ++w) {
                uint32_t bits = row[w];
                while (bits) {
                    const uint32_t j = w * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    best = min(best, label[j]);
                }
            }
            if (best < label[i]) {
                label[i] = best;
                changed = 1;
            }
        }
        __syncthreads();
        if (!changed) break;
    }
}

}  // namespace
}  // namespace pchase

extern "C" int pchase_miss_rates(const uint64_t *counts, uint32_t n_geoms, uint32_t n_points,
                                 const uint64_t *measured, float *rates_out,
                                 pchase_stream_t stream) {
    using namespace pchase;
    if (!counts || !measured || !rates_out)
        return set_last_error(PCHASE_EINVAL, "pchase_miss_rates: NULL argument");
    const uint64_t n = (uint64_t)n_geoms * n_points;
    if (n == 0) return PCHASE_OK;
    const unsigned blocks = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    miss_rates_kernel<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        counts, n_geoms, n_points, measured, rates_out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCHASE_OK : set_last_error(PCHASE_ECUDA, cudaGetErrorString(e));
}

extern "C" size_t pchase_answer_classes_work_bytes(uint32_t n_geoms) {
    const size_t words = (n_geoms + 31) / 32;
    return ((size_t)n_geoms * words * 4 + 255) & ~size_t(255);
}

extern "C" int pchase_answer_classes(const float *rates, uint32_t n_geoms, uint32_t n_points,
                                     double tol, uint32_t *rep_out, void *work,
                                     pchase_stream_t stream) {
    using namespace pchase;
    if (!rates || !rep_out || !work)
        return set_last_error(PCHASE_EINVAL, "pchase_answer_classes: NULL argument");
    if (n_geoms == 0) return PCHASE_OK;
    if (n_geoms > 65536)
        return set_last_error(PCHASE_ERANGE, "pchase_answer_classes: at most 65536 geometries");
    if (!(tol >= 0.0)) return set_last_error(PCHASE_EINVAL, "pchase_answer_classes: tol < 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t words = (n_geoms + 31) / 32;
    uint32_t *adj = static_cast<uint32_t *>(work);
    cudaError_t e = cudaMemsetAsync(adj, 0, (size_t)n_geoms * words * 4, st);
    if (e == cudaSuccess) {
        adjacency_kernel<<<n_geoms, 256, 0, st>>>(rates, n_geoms, n_points, tol, adj, words);
        components_kernel<<<1, 1024, 0, st>>>(adj, n_geoms, words, rep_out);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? PCHASE_OK : set_last_error(PCHASE_ECUDA, cudaGetErrorString(e));
}
