// noalloc.cu -- tu_fused_halfsweep_noalloc: one fused X half-sweep on caller
// buffers that never allocates device memory.
//
// Some callers cannot call cudaMalloc: a serving process whose device memory
// is fully budgeted by an admission controller or already held by another
// allocator (a framework's caching allocator), or a latency-critical loop in
// which cudaMalloc / cudaFree would synchronise the device. For them the
// scratch this half-sweep needs (the prepared partner vector, the FP64 own
// state, the reduction partials) lives in one file-scope __device__ array of
// fixed size, which every GPU that loads the library holds until the process
// exits. Every call shares that array; calls that overlap on the GPU race.
#include <cmath>
#include <mutex>

#include "tu_internal.cuh"

namespace {

using namespace tu;

constexpr int64_t kNaMaxRows = 65536;    // own users per call
constexpr int64_t kNaMaxCols = 1 << 20;  // partner users per call
constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 1024;       // blocks of the partner max reduction

// Scratch layout (byte offsets, every region 256-byte aligned).
constexpr size_t kOffPvec = 0;                                       // kNaMaxCols floats
constexpr size_t kOffLogU = kOffPvec + (size_t)kNaMaxCols * 4;       // kNaMaxRows doubles
constexpr size_t kOffEll = kOffLogU + (size_t)kNaMaxRows * 8;        // kNaMaxRows doubles
constexpr size_t kOffB2s = kOffEll + (size_t)kNaMaxRows * 8;         // kNaMaxRows floats
constexpr size_t kOffMpart = kOffB2s + (size_t)kNaMaxRows * 4;       // kNaMaxBlocks doubles
constexpr size_t kOffPart = kOffMpart + (size_t)kNaMaxBlocks * 8;    // kMaxPartials x 4 doubles
constexpr size_t kOffLmax = kOffPart + (size_t)kMaxPartials * 4 * 8;  // 1 double
constexpr size_t kOffResult = kOffLmax + 8;                           // 2 doubles
constexpr size_t kOffErr = kOffResult + 16;                           // 1 int
constexpr size_t kScratchBytes = kOffErr + 256;                       // 5,644,576 bytes (about 5.4 MiB)

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceScratch {
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  int num_sms = 0;
  bool ready = false;
};
std::mutex g_setup_mu;
DeviceScratch g_devices[64];

// Once per device, with that device current: resolve the array's device address.
tu_status setup_device(int dev, DeviceScratch* out) {
  if (dev < 0 || dev >= 64) return TU_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceScratch& d = g_devices[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return TU_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      return TU_ERR_CUDA;
    }
    d.base = static_cast<unsigned char*>(ptr);
    d.num_sms = sms;
    d.ready = true;
  }
  *out = d;
  return TU_OK;
}

// Device (or managed) memory of device `dev`: a buffer of another GPU would be
// read through a peer mapping, or fault where peer access is off.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// ell_c = log v_c + b_c / (2 sigma) (same rounding of b / (2 sigma) as a market), per-block maxima.
__global__ void k_na_prep_max(const float* __restrict__ log_v, const float* __restrict__ bias, float inv2s,
                              int64_t cols, double* __restrict__ mpart) {
  __shared__ double red[kNaThreads / 32];
  double mx = -INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cols; i += (int64_t)gridDim.x * blockDim.x) {
    const float b2s = bias ? (float)((double)bias[i] * (double)inv2s) : 0.0f;
    mx = fmax(mx, (double)log_v[i] + (double)b2s);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -INFINITY;
    for (int w = 0; w < kNaThreads / 32; ++w) b = fmax(b, red[w]);
    mpart[blockIdx.x] = b;
  }
}

// Prepared partner vector g_c = (ell_c - max ell) * log2(e), -inf padding.
__global__ void k_na_prep_write(const float* __restrict__ log_v, const float* __restrict__ bias, float inv2s,
                                int64_t cols, int64_t cols_pad, const double* __restrict__ mpart, int nparts,
                                float* __restrict__ pvec, double* __restrict__ lmax) {
  __shared__ double red[kNaThreads / 32];
  __shared__ double shift_s;
  double mx = -INFINITY;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) mx = fmax(mx, mpart[i]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -INFINITY;
    for (int w = 0; w < kNaThreads / 32; ++w) b = fmax(b, red[w]);
    if (!(b > -INFINITY && b < INFINITY)) b = 0.0;
    shift_s = b;
    if (blockIdx.x == 0) *lmax = b;
  }
  __syncthreads();
  const double shift = shift_s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cols_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v = -INFINITY;
    if (i < cols) {
      const float b2s = bias ? (float)((double)bias[i] * (double)inv2s) : 0.0f;
      v = (float)(((double)log_v[i] + (double)b2s - shift) * 1.4426950408889634);
    }
    pvec[i] = v;
  }
}

// Own side into the FP64 state; clears the error word before the half-sweep runs.
__global__ void k_na_own_in(const float* __restrict__ log_u_in, const float* __restrict__ bias, float inv2s,
                            int64_t rows, double* __restrict__ log_u, float* __restrict__ b2s, int* __restrict__ err) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *err = kErrNone;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
    log_u[i] = (double)log_u_in[i];
    if (b2s != nullptr) b2s[i] = bias ? (float)((double)bias[i] * (double)inv2s) : 0.0f;
  }
}

// New log u to the caller (FP32) and the FP64 residual reduction (block 0).
__global__ void k_na_finish(const double* __restrict__ log_u, int64_t rows, float* __restrict__ out,
                            const double* __restrict__ partials, int nparts, double* __restrict__ result) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)log_u[i];
  if (blockIdx.x != 0) return;
  __shared__ double s_max[kNaThreads], s_nf[kNaThreads];
  double mx = 0.0, nf = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    mx = fmax(mx, partials[4 * i + 0]);
    nf += partials[4 * i + 3];
  }
  s_max[threadIdx.x] = mx;
  s_nf[threadIdx.x] = nf;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + w]);
      s_nf[threadIdx.x] += s_nf[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    result[0] = s_max[0];
    result[1] = s_nf[0];
  }
}

int blocks_for(int64_t n, int num_sms) {
  int64_t g = (n + kNaThreads - 1) / kNaThreads;
  if (g > (int64_t)num_sms * 4) g = (int64_t)num_sms * 4;
  if (g > kNaMaxBlocks) g = kNaMaxBlocks;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

extern "C" tu_status tu_fused_halfsweep_noalloc(int64_t rows, int64_t cols, int64_t kp, const void* own_packed,
                                                const void* partner_packed, const float* own_bias,
                                                const double* own_mass, const float* own_log_u_in,
                                                const float* partner_bias, const float* partner_log_v, double sigma,
                                                float* own_log_u_out, double* residual_out, void* stream) {
  if (rows < 1 || cols < 1 || !(sigma > 0.0) || !(sigma < INFINITY)) return TU_ERR_INVALID_ARG;
  if (!own_packed || !partner_packed || !own_mass || !own_log_u_in || !partner_log_v || !own_log_u_out)
    return TU_ERR_INVALID_ARG;
  if (rows > kNaMaxRows || cols > kNaMaxCols) return TU_ERR_UNSUPPORTED;
  if (kp != 64 && kp != 128) return TU_ERR_UNSUPPORTED;
  if (((uintptr_t)own_packed | (uintptr_t)partner_packed) & 15u) return TU_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TU_ERR_CUDA;
  }
  const void* dev_ptrs[] = {own_packed, partner_packed, own_mass, own_log_u_in, partner_log_v, own_log_u_out,
                            own_bias, partner_bias};
  for (const void* p : dev_ptrs)
    if (p != nullptr && !on_device(p, dev)) return TU_ERR_INVALID_ARG;
  if (!device_supported(dev)) return TU_ERR_UNSUPPORTED;
  DeviceScratch ds;
  tu_status st = setup_device(dev, &ds);
  if (st != TU_OK) return st;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* pvec = reinterpret_cast<float*>(ds.base + kOffPvec);
  double* log_u = reinterpret_cast<double*>(ds.base + kOffLogU);
  double* ell = reinterpret_cast<double*>(ds.base + kOffEll);
  float* b2s = own_bias ? reinterpret_cast<float*>(ds.base + kOffB2s) : nullptr;
  double* mpart = reinterpret_cast<double*>(ds.base + kOffMpart);
  double* partials = reinterpret_cast<double*>(ds.base + kOffPart);
  double* lmax = reinterpret_cast<double*>(ds.base + kOffLmax);
  double* result = reinterpret_cast<double*>(ds.base + kOffResult);
  int* err = reinterpret_cast<int*>(ds.base + kOffErr);
  const float inv2s = (float)(0.5 / sigma);
  const int64_t cols_pad = (cols + kFusedPartnerRows - 1) / kFusedPartnerRows * kFusedPartnerRows;

  const int g1 = blocks_for(cols, ds.num_sms);
  k_na_prep_max<<<g1, kNaThreads, 0, s>>>(partner_log_v, partner_bias, inv2s, cols, mpart);
  k_na_prep_write<<<blocks_for(cols_pad, ds.num_sms), kNaThreads, 0, s>>>(partner_log_v, partner_bias, inv2s, cols,
                                                                         cols_pad, mpart, g1, pvec, lmax);
  k_na_own_in<<<blocks_for(rows, ds.num_sms), kNaThreads, 0, s>>>(own_log_u_in, own_bias, inv2s, rows, log_u, b2s,
                                                                 err);
  if (cudaGetLastError() != cudaSuccess) return TU_ERR_CUDA;
  FusedRaw r;
  r.own16 = static_cast<const __nv_bfloat16*>(own_packed);
  r.rows = rows;
  r.par16 = static_cast<const __nv_bfloat16*>(partner_packed);
  r.cols = cols;
  r.kp = kp;
  r.sigma = sigma;
  r.g = pvec;
  r.lmax = lmax;
  r.b2s = b2s;
  r.mass = own_mass;
  r.log_u = log_u;
  r.ell = ell;
  r.partials = partials;
  r.err = err;
  r.residual = residual_out != nullptr ? kResidualExact : kResidualNone;
  int nparts = 0;
  if (launch_fused_halfsweep_raw(r, s, ds.num_sms, &nparts) != cudaSuccess) {
    cudaGetLastError();
    return TU_ERR_CUDA;
  }
  k_na_finish<<<blocks_for(rows, ds.num_sms), kNaThreads, 0, s>>>(log_u, rows, own_log_u_out, partials, nparts,
                                                                 result);
  if (cudaGetLastError() != cudaSuccess) return TU_ERR_CUDA;
  if (residual_out != nullptr) {
    double host_res[2] = {0.0, 0.0};
    int host_err = 0;
    if (cudaMemcpyAsync(host_res, result, sizeof(host_res), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&host_err, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return TU_ERR_CUDA;
    }
    if (host_err == kErrTimeout) return TU_ERR_TIMEOUT;
    if (host_err != kErrNone) return TU_ERR_CUDA;
    if (host_res[1] > 0.0) return TU_ERR_NONFINITE;
    *residual_out = host_res[0];
  }
  return TU_OK;
}
