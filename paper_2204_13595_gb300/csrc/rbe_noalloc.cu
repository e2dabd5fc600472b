// rbe_noalloc.cu -- structure factors rho(k) without any device allocation.
//
// Some callers cannot let this library allocate device memory: a host
// process whose GPU memory is owned in full by another allocator (a
// framework's caching allocator that has already reserved the device, or a
// service running under a fixed memory budget), or code on a path where an
// allocation call is not allowed or where cudaFree's implicit device
// synchronisation is not acceptable.  rbe_rho_noalloc serves them: it
// computes the structure factors of the context path with its per-block
// scratch in a file-scope device array that exists from module load to
// process exit.  The caller passes every input and output; nothing here calls
// cudaMalloc, cudaFree or an allocating library routine.
//
// Scratch: RBE_NOALLOC_BLOCKS x RBE_NOALLOC_PMAX double2 partial sums (2 MiB),
// held by every GPU that loads the library.  Every call rewrites all entries
// it later reads, so nothing has to start at zero; calls whose kernels
// overlap on the GPU (different streams, different host threads) share the
// array and race.
#include <mutex>

#include "rbe_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_TILE = 256;

static __device__ __align__(256) double2 g_rho_scratch[RBE_NOALLOC_BLOCKS * RBE_NOALLOC_PMAX];

// Device address of g_rho_scratch per device, looked up once per device with
// that device current (the host-side symbol is only a stand-in).  The cached
// address is not refreshed after cudaDeviceReset: a process that resets a
// device must not call rbe_rho_noalloc on it again.
std::mutex g_mu;
double2* g_scratch_ptr[256];
bool g_scratch_ok[256];

// Block b sums q_j exp(i k_l . r_j) over atoms [b*chunk, (b+1)*chunk) for
// every l; thread t owns k_l for l = t, t + blockDim, ...  The phase
// t = (m . x_wrapped)/L is formed in FP64, reduced to [-1/2, 1/2] by rint
// and evaluated with sincospi; the block partials are summed serially in
// block order.  This is not the context path's arithmetic (which takes the
// phase from the 32-bit fixed-point codes and a table with a Taylor series,
// and sums in another order): the two agree to rounding, about 1e-13 of
// sum |q|, not bit for bit, and the rounding of the FP64 phase grows with
// |m . x| / L.
__global__ void __launch_bounds__(NA_THREADS) k_rho_noalloc(int n, int chunk, double L, double invL, int P,
                                                            const double* __restrict__ pos,
                                                            const double* __restrict__ q,
                                                            const int32_t* __restrict__ m,
                                                            double2* __restrict__ part)
{
    __shared__ double4_32a tile[NA_TILE];
    const int b0 = blockIdx.x * chunk;
    const int b1 = min(n, b0 + chunk);
    for (int l0 = 0; l0 < P; l0 += blockDim.x) {
        const int l = l0 + threadIdx.x;
        const bool act = l < P;
        const double mx = act ? m[3 * l] : 0.0, my = act ? m[3 * l + 1] : 0.0, mz = act ? m[3 * l + 2] : 0.0;
        double re = 0.0, im = 0.0;
        for (int t0 = b0; t0 < b1; t0 += NA_TILE) {
            const int cnt = min(NA_TILE, b1 - t0);
            __syncthreads();
            for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
                const int j = t0 + k;
                double xw, yw, zw;
                uint32_t s;
                wrap_fixed(pos[3 * j], invL, L, xw, s);
                wrap_fixed(pos[3 * j + 1], invL, L, yw, s);
                wrap_fixed(pos[3 * j + 2], invL, L, zw, s);
                tile[k] = make_double4_32a(xw, yw, zw, q[j]);
            }
            __syncthreads();
            if (act) {
                for (int k = 0; k < cnt; ++k) {
                    const double4_32a p = tile[k];
                    double t = (mx * p.x + my * p.y + mz * p.z) * invL;
                    t -= rint(t);
                    double sn, cs;
                    sincospi(2.0 * t, &sn, &cs);
                    re += p.w * cs;
                    im += p.w * sn;
                }
            }
        }
        if (act) part[(size_t)blockIdx.x * P + l] = make_double2(re, im);
    }
}

// Fixed-order sum of the block partials.
__global__ void __launch_bounds__(NA_THREADS) k_rho_noalloc_sum(int nblk, int P, const double2* __restrict__ part,
                                                                double* __restrict__ rho)
{
    const int l = blockIdx.x * NA_THREADS + threadIdx.x;
    if (l >= P) return;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < nblk; ++b) {
        const double2 v = part[(size_t)b * P + l];
        re += v.x;
        im += v.y;
    }
    rho[2 * l] = re;
    rho[2 * l + 1] = im;
}

}  // namespace

extern "C" int rbe_rho_noalloc(int n, const double* pos, const double* q, double box_L, int P, const int32_t* m,
                               double* rho, void* cuda_stream)
{
    if (n < 0 || !(box_L > 0.0) || P < 1 || !m || !rho || (n > 0 && (!pos || !q))) return RBE_EINVAL;
    if (P > RBE_NOALLOC_PMAX) return RBE_ELIMIT;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return RBE_ECUDA;
    double2* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ok[dev]) {
            // set-up on the first call on this device (current device)
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_rho_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return RBE_ECUDA;
            }
            g_scratch_ptr[dev] = static_cast<double2*>(p);
            g_scratch_ok[dev] = true;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int blocks = (n + NA_TILE - 1) / NA_TILE;
    blocks = blocks < 1 ? 1 : (blocks > RBE_NOALLOC_BLOCKS ? RBE_NOALLOC_BLOCKS : blocks);
    const int chunk = (n + blocks - 1) / blocks;
    const int threads = ((P < NA_THREADS ? P : NA_THREADS) + 31) / 32 * 32;
    // cudaGetLastError also returns (and clears) an error that an earlier
    // launch of the caller's left pending; such an error is reported here as
    // RBE_ECUDA
    k_rho_noalloc<<<blocks, threads, 0, st>>>(n, chunk, box_L, 1.0 / box_L, P, pos, q, m, scratch);
    if (cudaGetLastError() != cudaSuccess) return RBE_ECUDA;
    k_rho_noalloc_sum<<<(P + NA_THREADS - 1) / NA_THREADS, NA_THREADS, 0, st>>>(blocks, P, scratch, rho);
    if (cudaGetLastError() != cudaSuccess) return RBE_ECUDA;
    return RBE_OK;
}
