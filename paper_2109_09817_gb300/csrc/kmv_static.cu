// gp_kmatmul_noalloc: K-hat V for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc or any allocating routine: code that
// runs inside a memory pool they do not own, a process whose device memory
// is reserved up front by another framework, or a real-time loop where an
// allocation (and the device synchronisation that cudaFree implies) is not
// allowed.  This entry point does the same product as gp_kmatmul with
// GP_FP32_PLAIN arithmetic, but keeps its scratch (column means, prepared
// features, row norms) in one file-scope __device__ array of fixed size, and
// takes the stream directly instead of a context (a context owns a growable
// workspace).  It calls no cudaMalloc, cudaFree, cudaMallocHost or other
// allocating routine; the lengthscales travel as kernel arguments.
//
// Limits: N * round_up(d, 32) <= GP_NOALLOC_MAX_FEATURES floats, N <=
// GP_NOALLOC_MAX_ROWS, d <= GP_NOALLOC_MAX_D, 1 <= t <= 512.  Every GPU that
// loads the library holds the array until the process exits.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "gp_internal.cuh"

namespace {

constexpr int64_t kMaxFeat = GP_NOALLOC_MAX_FEATURES;
constexpr int64_t kMaxRows = GP_NOALLOC_MAX_ROWS;
constexpr int kMaxD = GP_NOALLOC_MAX_D;
constexpr int kMeanBlocks = 64;
// layout: [mean partials kMeanBlocks x kMaxD doubles][mean kMaxD doubles]
//         [features kMaxFeat floats][norms kMaxRows floats]
constexpr size_t kOffPart = 0;
constexpr size_t kOffMean = kOffPart + sizeof(double) * kMeanBlocks * kMaxD;
constexpr size_t kOffFeat = kOffMean + sizeof(double) * kMaxD;
constexpr size_t kOffNorm = kOffFeat + sizeof(float) * kMaxFeat;
constexpr size_t kScratchBytes = kOffNorm + sizeof(float) * kMaxRows;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host-side address of the array on each device, set once per device.
std::mutex g_mu;
void* g_addr[64] = {};

constexpr float kC1f = 0.69314718055994530942f;   // ln 2
constexpr float kC2f = 0.16014921423310860f;      // (ln 2)^2 / 3
constexpr double kScale = 2.23606797749978969640917366873 * 1.44269504088896340735992468100;

struct Scales {
  double v[kMaxD];   // sqrt5 log2e / l_j
};

__global__ void na_mean_partial(const float* __restrict__ X, int64_t n, int d,
                                double* __restrict__ part) {
  // block b sums rows b, b + nblk, ... ; thread j handles feature j
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double acc = 0.0;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) acc += (double)X[r * d + j];
    part[(int64_t)blockIdx.x * kMaxD + j] = acc;
  }
}

__global__ void na_mean_final(const double* __restrict__ part, int nblk, int d, int64_t n,
                              double* __restrict__ mu) {
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * kMaxD + j];
    mu[j] = s / (double)n;
  }
}

// one warp per padded row: x~ = (x - mu) sqrt5 log2e / l, |x~|^2
__global__ void na_prep(const float* __restrict__ X, int64_t n, int d, int64_t n_pad, int d_pad,
                        const double* __restrict__ mu, const Scales sc, float* __restrict__ xt,
                        float* __restrict__ nrm) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n_pad) return;
  double acc = 0.0;
  for (int j = lane; j < d_pad; j += 32) {
    float v = 0.f;
    if (row < n && j < d) v = (float)(((double)X[row * d + j] - mu[j]) * sc.v[j]);
    xt[row * d_pad + j] = v;
    acc += (double)v * v;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) nrm[row] = (float)acc;
}

__global__ void na_init(const float* __restrict__ V, int t, int64_t n, float* __restrict__ out,
                        float sigma2) {
  const int64_t total = n * t;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = sigma2 * V[i];
}

// 64-row x 64-column tiles, 256 threads (4 x 4 entries each); the K tile goes
// through shared memory to the contraction with up to 16 vectors per pass.
constexpr int TB = 64;
constexpr int KC = 32;
__global__ void __launch_bounds__(256)
na_kmv(const float* __restrict__ xt, const float* __restrict__ nrm, int64_t n, int d_pad,
       const float* __restrict__ V, int t, int c0, float* __restrict__ out, float s) {
  __shared__ float sA[TB][KC + 1];
  __shared__ float sB[TB][KC + 1];
  __shared__ float sK[TB][TB + 1];
  __shared__ float sV[16][TB + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * TB;
  const int tc = min(16, t - c0);
  // thread (ty, tx): rows ty*4 .. +4; output columns: vector tx (one per thread)
  float o[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t col0 = 0; col0 < n; col0 += TB) {
    float acc[4][4] = {};
    for (int k0 = 0; k0 < d_pad; k0 += KC) {
      __syncthreads();
      for (int i = tid; i < TB * KC; i += 256) {
        const int r = i / KC, k = i % KC;
        sA[r][k] = xt[(row0 + r) * d_pad + k0 + k];
        sB[r][k] = xt[(col0 + r) * d_pad + k0 + k];
      }
      __syncthreads();
      for (int k = 0; k < KC; ++k)
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(sA[ty * 4 + i][k], sB[tx * 4 + j][k], acc[i][j]);
    }
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const int64_t a = row0 + ty * 4 + i, b = col0 + tx * 4 + j;
        float u2 = fmaxf(fmaf(-2.f, acc[i][j], nrm[a] + nrm[b]), 0.f);
        float u, e;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(u) : "f"(u2));
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-u));
        float kv = fmaf(u2, kC2f, fmaf(u, kC1f, 1.f)) * e;
        if (a == b) kv = 1.f;
        sK[ty * 4 + i][tx * 4 + j] = kv;
      }
    for (int i = tid; i < 16 * TB; i += 256) {
      const int c = i / TB, b = i % TB;
      const int64_t col = col0 + b;
      sV[c][b] = (c < tc && col < n) ? V[(int64_t)(c0 + c) * n + col] : 0.f;
    }
    __syncthreads();
    for (int b = 0; b < TB; ++b)
      for (int i = 0; i < 4; ++i) o[i] = fmaf(sK[ty * 4 + i][b], sV[tx][b], o[i]);
  }
  if (tx < tc)
    for (int i = 0; i < 4; ++i) {
      const int64_t a = row0 + ty * 4 + i;
      if (a < n) out[(int64_t)(c0 + tx) * n + a] += s * o[i];
    }
}

}  // namespace

extern "C" int gp_kmatmul_noalloc(const float* X, int64_t N, int d, const gp_theta* theta,
                                  const float* V, int t, float* out, void* stream) {
  if (!X || !V || !out || !theta || !theta->lengthscale || N <= 0 || d <= 0 || t < 1 || t > 512)
    return GP_EINVAL;
  if (d > kMaxD || N > kMaxRows) return GP_EINVAL;
  const int d_pad = (d + 31) / 32 * 32;
  const int64_t n_pad = (N + TB - 1) / TB * TB;
  if (n_pad * d_pad > kMaxFeat || n_pad > kMaxRows) return GP_EINVAL;
  if (!(theta->outputscale > 0.0) || !(theta->sigma2 > 0.0)) return GP_EINVAL;
  Scales sc;
  for (int j = 0; j < d; ++j) {
    if (!(theta->lengthscale[j] > 0.0) || !std::isfinite(theta->lengthscale[j])) return GP_EINVAL;
    sc.v[j] = kScale / theta->lengthscale[j];
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ECUDA;
  unsigned char* base = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
        cudaGetLastError();
        return GP_ECUDA;
      }
      g_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_addr[dev]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* part = reinterpret_cast<double*>(base + kOffPart);
  double* mu = reinterpret_cast<double*>(base + kOffMean);
  float* xt = reinterpret_cast<float*>(base + kOffFeat);
  float* nrm = reinterpret_cast<float*>(base + kOffNorm);
  const int nblk = (int)std::min<int64_t>(kMeanBlocks, N);
  na_mean_partial<<<nblk, 256, 0, st>>>(X, N, d, part);
  na_mean_final<<<1, 256, 0, st>>>(part, nblk, d, N, mu);
  na_prep<<<(unsigned)((n_pad + 7) / 8), 256, 0, st>>>(X, N, d, n_pad, d_pad, mu, sc, xt, nrm);
  const unsigned gi = (unsigned)std::min<int64_t>((N * t + 255) / 256, 4096);
  na_init<<<std::max(1u, gi), 256, 0, st>>>(V, t, N, out, (float)theta->sigma2);
  const unsigned gk = (unsigned)(n_pad / TB);
  for (int c0 = 0; c0 < t; c0 += 16)
    na_kmv<<<gk, 256, 0, st>>>(xt, nrm, N, d_pad, V, t, c0, out, (float)theta->outputscale);
  return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ECUDA;
}
