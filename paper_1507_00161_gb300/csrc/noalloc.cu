// H_eff psi without device allocation.
//
// Some callers cannot call cudaMalloc during a product: a process whose device memory is
// owned and budgeted up front by another allocator (a serving framework that reserved
// the GPU), code that must not pay the implicit device synchronisation an allocation or
// a free can cause, or code with no way to recover from a failed allocation.  This file
// gives them dmrg_heff_apply_noalloc: the same FP64 two-stage product as dmrg_heff_apply,
// with the stage-1 intermediate held in a fixed file-scope device array instead of a
// buffer the library allocates.
#include <mutex>

#include "common.h"

namespace {

// 2,097,152 doubles = 16 MiB (kScratchElems, common.h), held by every GPU that loads the
// library until exit
static __device__ __align__(256) double g_heff_scratch[dmrg::kScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of the array on the current device.  In host code the symbol is only a
// host-side stand-in, so the address is looked up once per device, with that device
// current, and cached.
double* scratch_on_current_device() {
  int dev = -1;
  DMRG_CUDA(cudaGetDevice(&dev));
  DMRG_REQUIRE(dev >= 0 && dev < kMaxDevices, DMRG_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_heff_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw dmrg::Error(DMRG_ECUDA, std::string("cudaGetSymbolAddress of the H_eff scratch: ") +
                                        cudaGetErrorString(e));
    g_addr[dev] = static_cast<double*>(p);
  }
  return g_addr[dev];
}

}  // namespace

extern "C" int dmrg_heff_apply_noalloc(dmrg_ctx* c, int32_t p, const double* x, double* y) {
  if (!c) return DMRG_EINVAL;
  try {
    DMRG_REQUIRE(x && y && x != y, DMRG_EINVAL, "bad vectors");
    dmrg::HeffView v;
    DMRG_REQUIRE(dmrg::heff_view(c, p, &v), DMRG_EINVAL,
                 "the superblock at this position is not set up: call dmrg_psi_layout or "
                 "dmrg_heff_apply at this position first (those calls allocate)");
    DMRG_REQUIRE(v.t_elems <= dmrg::kScratchElems, DMRG_EINVAL,
                 "this product needs " + std::to_string(v.t_elems) +
                     " doubles of intermediate storage; the allocation-free entry point is "
                     "limited to 2097152 doubles (16 MiB)");
    DMRG_REQUIRE(v.lists_ready, DMRG_EINVAL,
                 "the superblock at this position is not set up: call dmrg_psi_layout or "
                 "dmrg_heff_apply at this position first (those calls allocate)");
    int dev = -1;
    DMRG_CUDA(cudaGetDevice(&dev));
    DMRG_REQUIRE(v.device < 0 || dev == v.device, DMRG_EINVAL,
                 "the current device is not the one the context was created on; make it "
                 "current before this call");
    double* T = scratch_on_current_device();
    // every element of the intermediate is written by stage 1 before stage 2 reads it;
    // the output is cleared here because blocks without terms receive no stage-2 task
    DMRG_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * v.size, v.stream));
    dmrg::Bases<double> b{};
    b.p[dmrg::B_LOPS] = const_cast<double*>(v.L);
    b.p[dmrg::B_ROPS] = const_cast<double*>(v.R);
    b.p[dmrg::B_X] = const_cast<double*>(x);
    b.p[dmrg::B_Y] = y;
    b.p[dmrg::B_T] = T;
    dmrg::run_gemm_tasks<double>(*v.st1, b, 1, v.stream);
    dmrg::run_gemm_tasks<double>(*v.st2, b, 1, v.stream);
    DMRG_CUDA(cudaStreamSynchronize(v.stream));
    return DMRG_OK;
  } catch (const dmrg::Error& e) {
    dmrg::set_error(c, e.what());
    return e.code;
  } catch (const std::exception& e) {
    dmrg::set_error(c, e.what());
    return DMRG_EINVAL;
  }
}
