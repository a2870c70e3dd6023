// One-shot force evaluation that allocates nothing.
//
// Some callers cannot call cudaMalloc: allocator-free embedded runtimes,
// and host programs that hand out every byte of device memory from their
// own pool, where an allocation behind their back would fail or break
// their accounting.  bdm_forces_noalloc serves them: it runs the same grid
// build and force kernels as bdm_step, on caller-owned input and output
// buffers, with all of its working memory in one file-scope device array of
// fixed size (below).  Every GPU that loads this library keeps that array
// until the process exits.  The call waits for its stream (it reads the
// device error word before it gathers the results), so it must not be
// recorded into a CUDA stream capture.
#include <mutex>

#include "kernels.cuh"

namespace bdm {
namespace {

constexpr int64_t kMaxAgents = 16384;      // agents per call
constexpr int64_t kMaxBoxes = 1 << 17;     // grid boxes per call
constexpr int kMaxDevices = 64;

constexpr size_t up(size_t b) { return (b + 255) / 256 * 256; }

// Byte offsets of the pieces inside the scratch array.
constexpr size_t kM = (size_t)kMaxAgents;
constexpr size_t oSC = 0;
constexpr size_t oSS = oSC + up(sizeof(SimConst));
constexpr size_t oG = oSS + up(sizeof(SimState));
constexpr size_t oOrder = oG + up(sizeof(Globals));
constexpr size_t oBad = oOrder + up(sizeof(int32_t));
constexpr size_t oTstat = oBad + up(sizeof(unsigned long long));
constexpr size_t kTstatWords = kM / 2048 + 2;  // scan tiles of 2,048 slots
constexpr size_t oAX = oTstat + up(8 * kTstatWords);
constexpr size_t oAY = oAX + up(8 * kM);
constexpr size_t oAZ = oAY + up(8 * kM);
constexpr size_t oAD = oAZ + up(8 * kM);
constexpr size_t oAV = oAD + up(8 * kM);
constexpr size_t oAId = oAV + up(8 * kM);
constexpr size_t oASim = oAId + up(4 * kM);
constexpr size_t oAKey = oASim + up(4 * kM);
constexpr size_t oARank = oAKey + up(8 * kM);
constexpr size_t oAFlags = oARank + up(4 * kM);
constexpr size_t oANnz = oAFlags + up(kM);
constexpr size_t oCSlot = oANnz + up(kM);
constexpr size_t oCSim = oCSlot + up(4 * kM);
constexpr size_t oCKey = oCSim + up(4 * kM);
constexpr size_t oCR0 = oCKey + up(8 * kM);
constexpr size_t oCR1 = oCR0 + up(16 * kM);
constexpr size_t oCR64 = oCR1 + up(16 * kM);
constexpr size_t oCFlag = oCR64 + up(32 * kM);
constexpr size_t oCNnz = oCFlag + up(kM);
constexpr size_t oCStat = oCNnz + up(kM);
constexpr size_t oCF32 = oCStat + up(kM);
constexpr size_t oCF64 = oCF32 + up(16 * kM);
constexpr size_t oOvf = oCF64 + up(32 * kM);
constexpr size_t oTab = oOvf + up(4 * kM);
constexpr size_t kBytes = oTab + up(8 * (size_t)kMaxBoxes);

// The working memory: about 5 MB per GPU.
static __device__ __align__(256) unsigned char g_scratch[kBytes];

std::mutex g_mu;
unsigned char *g_ptr[kMaxDevices] = {};

template <typename T>
T *at(unsigned char *base, size_t off) {
  return reinterpret_cast<T *>(base + off);
}

}  // namespace
}  // namespace bdm

using namespace bdm;

extern "C" int bdm_forces_noalloc(const bdm_params *params, int64_t n, const double *xyz, const double *diameter,
                                  double *force, int32_t *nnz, void *cuda_stream) {
  if (!params || n < 0 || (n > 0 && (!xyz || !diameter || !force))) return BDM_E_INVAL;
  if (n > kMaxAgents) return BDM_E_CAPACITY;
  const bdm_params &p = *params;
  if (!(p.k >= 0) || !(p.gamma >= 0) || !(p.box_length >= 0) ||
      (p.precision != BDM_PREC_FP64 && p.precision != BDM_PREC_FP32_FORCE) || p.boundary == BDM_BOUNDARY_TOROIDAL)
    return BDM_E_INVAL;
  if (n == 0) return BDM_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BDM_E_CUDA;
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
      // Set-up, once per device, with that device current: the host-side
      // name of the array is not a device address; ask the runtime for it.
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return BDM_E_CUDA;
      }
      g_ptr[dev] = (unsigned char *)ptr;
    }
    base = g_ptr[dev];
  }
  DevCtx D{};
  D.sc = at<SimConst>(base, oSC);
  D.ss = at<SimState>(base, oSS);
  D.g = at<Globals>(base, oG);
  D.order = at<int32_t>(base, oOrder);
  D.n_sims = 1;
  D.total_slots = n;
  D.a.x = at<double>(base, oAX); D.a.y = at<double>(base, oAY); D.a.z = at<double>(base, oAZ);
  D.a.d = at<double>(base, oAD); D.a.v = at<double>(base, oAV);
  D.a.id = at<int32_t>(base, oAId); D.a.sim = at<int32_t>(base, oASim);
  D.a.pkey = at<uint64_t>(base, oAKey);
  D.a.rank = at<uint32_t>(base, oARank); D.a.flags = at<uint8_t>(base, oAFlags); D.a.nnz = at<uint8_t>(base, oANnz);
  D.c.slot = at<int32_t>(base, oCSlot); D.c.sim = at<int32_t>(base, oCSim); D.c.pkey = at<uint64_t>(base, oCKey);
  D.c.r0 = at<float4>(base, oCR0); D.c.r1 = at<float4>(base, oCR1); D.c.r64 = at<double4_32a>(base, oCR64);
  D.c.flag = at<uint8_t>(base, oCFlag); D.c.nnz = at<uint8_t>(base, oCNnz); D.c.stat = at<uint8_t>(base, oCStat);
  D.c.f32 = at<float4>(base, oCF32); D.c.f64 = at<double4_32a>(base, oCF64);
  D.tab.e = at<unsigned long long>(base, oTab);
  D.ovf = at<int32_t>(base, oOvf);
  D.tstat = at<unsigned long long>(base, oTstat);

  // Constants and cleared state: every call starts from zero, because the
  // array keeps whatever the previous call left in it.
  SimConst sc{};
  sc.k = p.k; sc.gamma = p.gamma; sc.adherence = p.adherence; sc.max_disp = p.max_displacement; sc.dt = p.dt;
  sc.box_length = p.box_length;
  sc.box_scale = 1.0;
  sc.kf = (float)p.k; sc.gammaf = (float)p.gamma;
  sc.adherence2f = (float)(p.adherence * p.adherence);
  sc.max_disp2f = (float)(p.max_displacement * p.max_displacement);
  sc.max_dispf = (float)p.max_displacement; sc.dtf = (float)p.dt;
  sc.precision = p.precision;
  sc.base = 0; sc.cap = n; sc.table_base = 0; sc.table_cap = kMaxBoxes;
  SimState ss{};
  ss.n = n;
  for (int a = 0; a < 3; ++a) { ss.bmin[a] = ~0ull; ss.bmax[a] = 0ull; }
  int32_t order0 = 0;
  cudaError_t e = cudaMemcpyAsync(D.sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(D.ss, &ss, sizeof(ss), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(D.order, &order0, sizeof(order0), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(D.g, 0, sizeof(Globals), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(D.tab.e, 0, sizeof(unsigned long long) * (size_t)kMaxBoxes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(D.tstat, 0, sizeof(unsigned long long) * kTstatWords, st);
  unsigned long long *bad = at<unsigned long long>(base, oBad);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0xFF, sizeof(unsigned long long), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BDM_E_CUDA;
  }
  // the first invalid row (non-finite value, diameter not > 0), if any
  launch_check_input(st, n, xyz, diameter, bad);
  launch_set_agents(D, st, 0, 0, n, n, xyz, diameter);
  launch_bbox(D, st);
  launch_params(D, st, 1);
  launch_count(D, st, 1);
  launch_scan(D, st);
  // the first iteration has no static agents (every agent is new), so the
  // symmetric force walk always applies; the placement zeroes its forces
  launch_place(D, st, 1, 1);
  launch_force(D, st, 0);
  // The grid's fit is known only on the device: read the error word before
  // the results are gathered into the caller's buffers.
  uint32_t err = 0;
  unsigned long long first_bad = ~0ull;
  e = cudaMemcpyAsync(&err, &D.g->err, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&first_bad, bad, sizeof(first_bad), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BDM_E_CUDA;
  }
  if (first_bad != ~0ull) return BDM_E_NONFINITE;
  // a non-finite input also makes the grid invalid (ERR_COORD): report it first
  if (err & ERR_NONFINITE) return BDM_E_NONFINITE;
  if (err & (ERR_TABLE | ERR_COORD)) return BDM_E_CAPACITY;
  if (err & ERR_TIMEOUT) return BDM_E_TIMEOUT;
  launch_gather_forces(D, st, 0, 0, n, force, nnz, nullptr);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BDM_E_CUDA;
  }
  return BDM_OK;
}
