// labs_enum.cu -- exhaustive search over skew-symmetric sequences of short odd length
// (L <= 63), the exact counterpart of the stochastic search for small L.
//
// The centre is fixed to s_c = +1 (negating a whole sequence keeps Eq. 4 and the ISL).
// Assignment a sets free variable i (i < c) to -1 when bit i of a is set.  Thread t
// owns the assignments whose high bits equal t and walks its low bits in Gray-code
// order, so consecutive assignments differ by one free variable; the even-lag C_k are
// updated by the change of one flip (positions j and q = L-1-j), and the ISL (Eq. 2)
// is the sum of their squares (odd lags vanish by Eq. 4).
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <mutex>

#include "labs_internal.cuh"
#include "labs_nvtx.h"

namespace labsgpu {

namespace {

constexpr int kEnumThreads = 128;
constexpr int kEnumMaxHighBits = 17;

__host__ __device__ inline int enum_low_bits(int free_bits)
{
    return free_bits > kEnumMaxHighBits ? free_bits - kEnumMaxHighBits : 0;
}

// +1 / -1 / 0 (outside 0..L-1) from the sequence mask (bit j set <=> s_j = -1).
__device__ __forceinline__ int sval(uint64_t mask, int L, int j)
{
    if (j < 0 || j >= L) return 0;
    return ((mask >> j) & 1ull) ? -1 : 1;
}

__device__ __forceinline__ uint64_t seq_mask(uint64_t a, int L, int n)
{
    const int c = n - 1;
    uint64_t m = 0;
    for (int j = 0; j < L; ++j) {
        int f = j <= c ? j : 2 * c - j;
        int bit = f < c ? (int)((a >> f) & 1ull) : 0;  // centre is +1
        if (j > c && ((j - c) & 1)) bit ^= 1;
        m |= (uint64_t)bit << j;
    }
    return m;
}

__global__ void __launch_bounds__(kEnumThreads) enum_kernel(int L, EnumPart* parts)
{
    __shared__ int Cs[32][kEnumThreads];  // even-lag C, Cs[m][thread] = C_{2m}
    __shared__ long long rmin[kEnumThreads];
    __shared__ unsigned long long rcnt[kEnumThreads], rfirst[kEnumThreads];
    const int n = (L + 1) / 2, c = n - 1;
    const int T = n - 1;
    const int b = enum_low_bits(T);
    const uint64_t high = (uint64_t)blockIdx.x * kEnumThreads + threadIdx.x;
    const uint64_t nhigh = 1ull << (T - b);
    long long best = LLONG_MAX;
    unsigned long long cnt = 0, first = 0;
    int* C = &Cs[0][threadIdx.x];
    if (high < nhigh) {
        uint64_t a = high << b;
        uint64_t mask = seq_mask(a, L, n);
        long long isl = 0;
        for (int m = 1; m < n; ++m) {
            int d = 0;
            for (int j = 0; j + 2 * m < L; ++j) d += sval(mask, L, j) * sval(mask, L, j + 2 * m);
            C[m * kEnumThreads] = d;
            isl += (long long)d * d;
        }
        best = isl;
        cnt = 1;
        first = a;
        const uint64_t steps = 1ull << b;
        for (uint64_t t = 1; t < steps; ++t) {
            const int j = __ffsll((long long)t) - 1;  // Gray code: bit j changes
            const int q = L - 1 - j;
            const int sj = sval(mask, L, j);
            isl = 0;
            for (int m = 1; m < n; ++m) {
                const int k = 2 * m;
                const int up = (j + k == q) ? 0 : sval(mask, L, j + k);
                const int dC = -4 * sj * (up + sval(mask, L, j - k));
                const int cm = C[m * kEnumThreads] + dC;
                C[m * kEnumThreads] = cm;
                isl += (long long)cm * cm;
            }
            mask ^= (1ull << j) | (1ull << q);
            a ^= 1ull << j;
            if (isl < best) {
                best = isl;
                cnt = 1;
                first = a;
            } else if (isl == best) {
                cnt += 1;
                if (a < first) first = a;
            }
        }
    }
    (void)c;
    rmin[threadIdx.x] = best;
    rcnt[threadIdx.x] = cnt;
    rfirst[threadIdx.x] = first;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long m = LLONG_MAX;
        unsigned long long k = 0, f = 0;
        for (int t = 0; t < kEnumThreads; ++t) {
            if (rcnt[t] == 0) continue;
            if (rmin[t] < m) {
                m = rmin[t];
                k = rcnt[t];
                f = rfirst[t];
            } else if (rmin[t] == m) {
                k += rcnt[t];
                if (rfirst[t] < f) f = rfirst[t];
            }
        }
        parts[blockIdx.x].min_isl = m;
        parts[blockIdx.x].count = k;
        parts[blockIdx.x].first = f;
    }
}

__global__ void enum_reduce_kernel(const EnumPart* parts, int nparts, EnumPart* out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long m = LLONG_MAX;
    unsigned long long k = 0, f = 0;
    for (int t = 0; t < nparts; ++t) {
        if (parts[t].count == 0) continue;
        if (parts[t].min_isl < m) {
            m = parts[t].min_isl;
            k = parts[t].count;
            f = parts[t].first;
        } else if (parts[t].min_isl == m) {
            k += parts[t].count;
            if (parts[t].first < f) f = parts[t].first;
        }
    }
    out->min_isl = m;
    out->count = k;
    out->first = f;
}

}  // namespace

int enum_blocks(int L)
{
    const int n = (L + 1) / 2;
    const int T = n - 1;
    const uint64_t nhigh = 1ull << (T - enum_low_bits(T));
    return (int)((nhigh + kEnumThreads - 1) / kEnumThreads);
}

// Scratch: one EnumPart per block plus the final result.
size_t enum_scratch_bytes(int L)
{
    return sizeof(EnumPart) * (size_t)(enum_blocks(L) + 1);
}

int enum_run(int L, EnumPart* scratch, void* stream, EnumPart* host_out)
{
    const int blocks = enum_blocks(L);
    cudaStream_t s = (cudaStream_t)stream;
    enum_kernel<<<blocks, kEnumThreads, 0, s>>>(L, scratch);
    enum_reduce_kernel<<<1, 32, 0, s>>>(scratch, blocks, scratch + blocks);
    if (cudaGetLastError() != cudaSuccess) return LABS_ECUDA;
    if (cudaMemcpyAsync(host_out, scratch + blocks, sizeof(EnumPart), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LABS_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LABS_ECUDA;
    return LABS_OK;
}

// ------------------------------------------------ allocation-free variant
//
// labs_enumerate_noalloc runs the same two kernels with their scratch (the per-block
// partial results and the final result) in the file-scope array below instead of a
// caller buffer.  The array is part of the library image: every GPU that loads the
// library holds its kNoAllocParts * 32 bytes (33,280 bytes) until the process exits.
// Host code cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device
// current) and keeps it per device.  A device reset (cudaDeviceReset) unloads the
// module and invalidates a kept address: a call whose CUDA work fails drops the kept
// address of its device, and the next call looks it up again.
constexpr int kNoAllocParts = 1040;  // enum_blocks(63) + 1 = 1025 fit
constexpr int kNoAllocDevices = 64;
static __device__ __align__(256) EnumPart g_noalloc_scratch[kNoAllocParts];

namespace {
std::mutex g_noalloc_mutex;
EnumPart* g_noalloc_addr[kNoAllocDevices] = {};
}  // namespace

}  // namespace labsgpu

extern "C" int labs_enumerate_noalloc(int32_t L, int64_t* min_isl, uint64_t* count, uint64_t* first_assignment,
                                      void* cuda_stream)
{
    LABS_API_RANGE();
    using namespace labsgpu;
    if (L < 3 || L > 63 || (L & 1) == 0) return LABS_EINVAL;
    const int blocks = enum_blocks(L);
    if (blocks + 1 > kNoAllocParts) return LABS_ENOMEM;  // needs more scratch than the static array holds
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LABS_ECUDA;
    if (dev < 0 || dev >= kNoAllocDevices) return LABS_EINVAL;
    EnumPart* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (g_noalloc_addr[dev] == nullptr) {
            void* addr = nullptr;
            if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || addr == nullptr) return LABS_ECUDA;
            g_noalloc_addr[dev] = static_cast<EnumPart*>(addr);
        }
        scratch = g_noalloc_addr[dev];
    }
    auto forget = [dev]() {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        g_noalloc_addr[dev] = nullptr;
    };
    // The array keeps the previous call's contents; clear the part this call uses.
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (cudaMemsetAsync(scratch, 0, sizeof(EnumPart) * (size_t)(blocks + 1), s) != cudaSuccess) {
        forget();
        return LABS_ECUDA;
    }
    EnumPart r;
    const int rc = enum_run(L, scratch, cuda_stream, &r);
    if (rc) {
        if (rc == LABS_ECUDA) forget();
        return rc;
    }
    if (min_isl) *min_isl = r.min_isl;
    if (count) *count = r.count;
    if (first_assignment) *first_assignment = r.first;
    return LABS_OK;
}
