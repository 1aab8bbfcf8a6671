// Launch wrappers and the registry of compiled (element, order, quadrature, model)
// kernel instances.
#pragma once
#include <type_traits>
#include <vector>

#include "ldg_kernels.cuh"

namespace ldg {

// Process-wide count of kernel launches issued by this library.
long long& launch_counter();
inline void count_launch() { ++launch_counter(); }

typedef cudaError_t (*StageFn)(int mode, const KArgs& a, cudaStream_t s);

struct KernelSet {
  int etype, p, nq, model;
  StageFn qstage;     // FP64 compute. Diffusion models: MODE_R / MODE_HOM; null otherwise
  StageFn residual;   // FP64 compute. MODE_R / MODE_HOM (linear models) / MODE_JV (nonlinear models)
  StageFn qstage32;   // FP32 compute, MODE_HOM (diffusion models); null otherwise
  StageFn residual32; // FP32 compute, MODE_HOM (linear) / MODE_JV (nonlinear): the Krylov J.v
  int ne_q, ne_r, ne_j, smem_q, smem_r, smem_j;
};

template <class EL, class MD, int MODE, class R> cudaError_t launch_res1(const KArgs& a, cudaStream_t s) {
  typedef RLayout<EL, MD, MODE, R> L;
  static const cudaError_t attr = cudaFuncSetAttribute(k_residual<EL, MD, MODE, R>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
  if (attr != cudaSuccess) return attr;
  if (a.E <= 0) return cudaSuccess;
  int grid = (a.E + L::NE - 1) / L::NE;
  k_residual<EL, MD, MODE, R><<<grid, 256, L::SMEM, s>>>(a);
  count_launch();
  return cudaGetLastError();
}
template <class EL, class MD, int MODE, class R> cudaError_t launch_q1(const KArgs& a, cudaStream_t s) {
  typedef QLayout<EL, MD, R> L;
  static const cudaError_t attr = cudaFuncSetAttribute(k_qstage<EL, MD, MODE, R>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
  if (attr != cudaSuccess) return attr;
  if (a.E <= 0) return cudaSuccess;
  int grid = (a.E + L::NE - 1) / L::NE;
  k_qstage<EL, MD, MODE, R><<<grid, 256, L::SMEM, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <class EL, class MD, class R> cudaError_t stage_res(int mode, const KArgs& a, cudaStream_t s) {
  if constexpr (MD::LINEAR) {
    if (mode == MODE_R) return launch_res1<EL, MD, MODE_R, R>(a, s);
    if (mode == MODE_HOM) return launch_res1<EL, MD, MODE_HOM, R>(a, s);
  } else {
    if (mode == MODE_R) return launch_res1<EL, MD, MODE_R, R>(a, s);
    if (mode == MODE_JV) return launch_res1<EL, MD, MODE_JV, R>(a, s);
  }
  return cudaErrorInvalidValue;
}
// FP32-compute stages: only the J.v modes are instantiated (the Newton residual stays FP64)
template <class EL, class MD> cudaError_t stage_res32(int mode, const KArgs& a, cudaStream_t s) {
  if constexpr (MD::LINEAR) {
    if (mode == MODE_HOM) return launch_res1<EL, MD, MODE_HOM, float>(a, s);
  } else {
    if (mode == MODE_JV) return launch_res1<EL, MD, MODE_JV, float>(a, s);
  }
  return cudaErrorInvalidValue;
}
template <class EL, class MD> cudaError_t stage_q32(int mode, const KArgs& a, cudaStream_t s) {
  if (mode == MODE_HOM) return launch_q1<EL, MD, MODE_HOM, float>(a, s);
  return cudaErrorInvalidValue;
}

template <class EL, class MD, class R> cudaError_t stage_q(int mode, const KArgs& a, cudaStream_t s) {
  if (mode == MODE_R) return launch_q1<EL, MD, MODE_R, R>(a, s);
  if (mode == MODE_HOM) return launch_q1<EL, MD, MODE_HOM, R>(a, s);
  return cudaErrorInvalidValue;
}

template <class EL, class MD> void add_set(std::vector<KernelSet>& reg, int etype) {
  KernelSet k;
  k.etype = etype; k.p = EL::P; k.nq = EL::NQ; k.model = MD::KIND;
  k.residual = &stage_res<EL, MD, double>;
  k.residual32 = &stage_res32<EL, MD>;
  k.ne_r = RLayout<EL, MD, MODE_R, double>::NE;
  k.smem_r = RLayout<EL, MD, MODE_R, double>::SMEM;
  if constexpr (MD::HASQ) {
    k.qstage = &stage_q<EL, MD, double>;
    k.qstage32 = &stage_q32<EL, MD>;
    k.ne_q = QLayout<EL, MD, double>::NE;
    k.smem_q = QLayout<EL, MD, double>::SMEM;
    k.ne_j = RLayout<EL, MD, MODE_HOM, double>::NE;
    k.smem_j = RLayout<EL, MD, MODE_HOM, double>::SMEM;
  } else {
    k.qstage = nullptr;
    k.qstage32 = nullptr;
    k.ne_q = 0; k.smem_q = 0;
    k.ne_j = RLayout<EL, MD, MODE_JV, double>::NE;
    k.smem_j = RLayout<EL, MD, MODE_JV, double>::SMEM;
  }
  reg.push_back(k);
}

void register_tri(std::vector<KernelSet>& reg);
void register_quad(std::vector<KernelSet>& reg);
void register_hex(std::vector<KernelSet>& reg);

}  // namespace ldg
