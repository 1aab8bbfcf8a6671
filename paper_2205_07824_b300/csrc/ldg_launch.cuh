// Launch wrappers and the registry of compiled (element, order, quadrature, model)
// kernel instances.
#pragma once
#include <atomic>
#include <type_traits>
#include <vector>

#include "ldg_kernels.cuh"

namespace ldg {

// Process-wide count of kernel launches issued by this library (host threads driving
// different contexts may launch at once).
std::atomic<long long>& launch_counter();
inline void count_launch() { launch_counter().fetch_add(1, std::memory_order_relaxed); }

typedef cudaError_t (*StageFn)(int mode, const KArgs& a, cudaStream_t s);
// columns col0 .. col0 + BLK_KT - 1 of the element-diagonal blocks (models without q)
typedef cudaError_t (*BlockFn)(int col0, const KArgs& a, cudaStream_t s);
constexpr int BLK_KT = 8;

struct KernelSet {
  int etype, p, nq, model;
  int tile;           // tile variant (Tile0 .. Tile3)
  bool linear;        // linear model: J.v is the homogeneous operator (MODE_HOM)
  bool curved;        // curved elements (per-point geometry records)
  StageFn qstage;     // FP64 compute. Models with q: MODE_R / MODE_HOM; null otherwise
  StageFn residual;   // FP64 compute. MODE_R / MODE_HOM (linear models) / MODE_JV (nonlinear models)
  StageFn qstage32;   // FP32 compute, MODE_HOM (models with q); null otherwise
  StageFn residual32; // FP32 compute, MODE_HOM (linear) / MODE_JV (nonlinear): the Krylov J.v
  BlockFn blocks;     // (unused: FP64 blocks take one tangent per launch)
  BlockFn blocks32;   // FP32 block columns by BLK_KT-tangent dual numbers (models without q)
  int ne_q, ne_r, ne_j, smem_q, smem_r, smem_j;
};

template <class EL, class MD, class R, class TL> cudaError_t launch_blk(int col0, const KArgs& a, cudaStream_t s) {
  typedef BLayout<EL, MD, R, TL, BLK_KT> L;
  static const cudaError_t attr = cudaFuncSetAttribute(k_block_columns<EL, MD, R, TL, BLK_KT>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
  if (attr != cudaSuccess) return attr;
  if (a.E <= 0) return cudaSuccess;
  int grid = (a.E + L::NE - 1) / L::NE;
  k_block_columns<EL, MD, R, TL, BLK_KT><<<grid, 256, L::SMEM, s>>>(a, col0);
  count_launch();
  return cudaGetLastError();
}

template <class EL, class MD, int MODE, class R, class TL> cudaError_t launch_res1(const KArgs& a, cudaStream_t s) {
  typedef RLayout<EL, MD, MODE, R, TL> L;
  static const cudaError_t attr = cudaFuncSetAttribute(k_residual<EL, MD, MODE, R, TL>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
  if (attr != cudaSuccess) return attr;
  if (a.E <= 0) return cudaSuccess;
  int grid = (a.E + L::NE - 1) / L::NE;
  k_residual<EL, MD, MODE, R, TL><<<grid, 256, L::SMEM, s>>>(a);
  count_launch();
  return cudaGetLastError();
}
template <class EL, class MD, int MODE, class R, class TL> cudaError_t launch_q1(const KArgs& a, cudaStream_t s) {
  if constexpr (EL::CURVED) {
    typedef QLayoutC<EL, MD, R, TL> L;
    static const cudaError_t attr = cudaFuncSetAttribute(k_qstage_curved<EL, MD, MODE, R, TL>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
    if (attr != cudaSuccess) return attr;
    if (a.E <= 0) return cudaSuccess;
    int grid = (a.E + L::NE - 1) / L::NE;
    k_qstage_curved<EL, MD, MODE, R, TL><<<grid, 256, L::SMEM, s>>>(a);
    count_launch();
    return cudaGetLastError();
  }
  typedef QLayout<EL, MD, R, TL> L;
  static const cudaError_t attr = cudaFuncSetAttribute(k_qstage<EL, MD, MODE, R, TL>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
  if (attr != cudaSuccess) return attr;
  if (a.E <= 0) return cudaSuccess;
  int grid = (a.E + L::NE - 1) / L::NE;
  k_qstage<EL, MD, MODE, R, TL><<<grid, 256, L::SMEM, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <class EL, class MD, class R, class TL> cudaError_t stage_res(int mode, const KArgs& a, cudaStream_t s) {
  if constexpr (MD::LINEAR) {
    if (mode == MODE_R) return launch_res1<EL, MD, MODE_R, R, TL>(a, s);
    if (mode == MODE_HOM) return launch_res1<EL, MD, MODE_HOM, R, TL>(a, s);
  } else {
    if (mode == MODE_R) return launch_res1<EL, MD, MODE_R, R, TL>(a, s);
    if (mode == MODE_JV) return launch_res1<EL, MD, MODE_JV, R, TL>(a, s);
  }
  return cudaErrorInvalidValue;
}
// FP32-compute stages: only the J.v modes are instantiated (the Newton residual stays FP64)
template <class EL, class MD, class TL> cudaError_t stage_res32(int mode, const KArgs& a, cudaStream_t s) {
  if constexpr (MD::LINEAR) {
    if (mode == MODE_HOM) return launch_res1<EL, MD, MODE_HOM, float, TL>(a, s);
  } else {
    if (mode == MODE_JV) return launch_res1<EL, MD, MODE_JV, float, TL>(a, s);
  }
  return cudaErrorInvalidValue;
}
template <class EL, class MD, class TL> cudaError_t stage_q32(int mode, const KArgs& a, cudaStream_t s) {
  if (mode == MODE_HOM) return launch_q1<EL, MD, MODE_HOM, float, TL>(a, s);
  return cudaErrorInvalidValue;
}

template <class EL, class MD, class R, class TL> cudaError_t stage_q(int mode, const KArgs& a, cudaStream_t s) {
  if (mode == MODE_R) return launch_q1<EL, MD, MODE_R, R, TL>(a, s);
  if (mode == MODE_HOM) return launch_q1<EL, MD, MODE_HOM, R, TL>(a, s);
  return cudaErrorInvalidValue;
}

template <class TL> constexpr int tile_id() {
  return std::is_same<TL, Tile0>::value ? 0 : std::is_same<TL, Tile1>::value ? 1 : std::is_same<TL, Tile2>::value ? 2 : 3;
}

template <class EL, class MD, class TL = Tile0> void add_set(std::vector<KernelSet>& reg, int etype) {
  KernelSet k;
  k.etype = etype; k.p = EL::P; k.nq = EL::NQ; k.model = MD::KIND;
  k.tile = tile_id<TL>();
  k.linear = MD::LINEAR;
  k.curved = EL::CURVED;
  k.residual = &stage_res<EL, MD, double, TL>;
  k.residual32 = &stage_res32<EL, MD, TL>;
  k.ne_r = RLayout<EL, MD, MODE_R, double, TL>::NE;
  k.smem_r = RLayout<EL, MD, MODE_R, double, TL>::SMEM;
  if constexpr (MD::HASQ) {
    k.qstage = &stage_q<EL, MD, double, TL>;
    k.qstage32 = &stage_q32<EL, MD, TL>;
    if constexpr (EL::CURVED) {
      k.ne_q = QLayoutC<EL, MD, double, TL>::NE;
      k.smem_q = QLayoutC<EL, MD, double, TL>::SMEM;
    } else {
      k.ne_q = QLayout<EL, MD, double, TL>::NE;
      k.smem_q = QLayout<EL, MD, double, TL>::SMEM;
    }
    constexpr int JM = MD::LINEAR ? MODE_HOM : MODE_JV;
    k.ne_j = RLayout<EL, MD, JM, double, TL>::NE;
    k.smem_j = RLayout<EL, MD, JM, double, TL>::SMEM;
    k.blocks = nullptr;
    k.blocks32 = nullptr;
  } else {
    k.qstage = nullptr;
    k.qstage32 = nullptr;
    k.blocks = nullptr;
    if constexpr (EL::CURVED) k.blocks32 = nullptr;   // curved: one tangent per launch
    else k.blocks32 = &launch_blk<EL, MD, float, TL>;
    k.ne_q = 0; k.smem_q = 0;
    k.ne_j = RLayout<EL, MD, MODE_JV, double, TL>::NE;
    k.smem_j = RLayout<EL, MD, MODE_JV, double, TL>::SMEM;
  }
  reg.push_back(k);
}

// Registration of the compiled instances, one function per element family and tile.
template <class TL> void register_tri_t(std::vector<KernelSet>& reg);
template <class TL> void register_quad_t(std::vector<KernelSet>& reg);
template <class TL> void register_hex_t(std::vector<KernelSet>& reg);
template <class TL> void register_ns_t(std::vector<KernelSet>& reg);
template <class TL> void register_curved_scalar_t(std::vector<KernelSet>& reg);
template <class TL> void register_tet_t(std::vector<KernelSet>& reg);
template <class TL> void register_curved_gas_t(std::vector<KernelSet>& reg);
template <class TL> void register_curved_tri_t(std::vector<KernelSet>& reg);
void register_all(std::vector<KernelSet>& reg);

// Nodal J.v kernels of the linear models on affine quadrilaterals / hexahedra
// (ldg_linear.cuh): both stages, q of the direction stored in qbuf.
typedef cudaError_t (*LinFn)(const KArgs& a, void* qbuf, cudaStream_t s);
// The launcher for (dim, p, convection?, precision LDG_FP64 / LDG_FP32), or null. cart:
// every element is an axis-aligned box (diagonal J^{-1}, face normals along their axes).
LinFn lin_launcher(int dim, int p, bool conv, int prec, bool cart);
// The same on triangles (etype 0) and tetrahedra (etype 3), or null.
LinFn lin_simplex_launcher(int etype, int p, bool conv, int prec);
// The same hexahedron / quadrilateral kernels in double-float arithmetic (ldg_df.cuh).
LinFn lin_df_launcher(int dim, int p, bool conv, bool cart);

// Euler J.v with the element contractions on the tensor cores (ldg_tcjv.cu), affine
// quadrilaterals with p + 2 Gauss points: passes 3 (BF16 hi/lo splits) or 1 (BF16).
// img: the constant operand image of build_tcjv_image on the device; err: set to 1
// when a wait timed out (the affected outputs are NaN).
typedef cudaError_t (*TcJvFn)(const KArgs& a, const unsigned char* img, int passes, int* err, cudaStream_t s);
TcJvFn tcjv_launcher(int p);   // p = 1..4, else null
// The constant operands (basis, derivative, face, lift and mass matrices as BF16 hi/lo
// images in the kernel's shared-memory layout) from the tensor element's FP64 blob.
bool build_tcjv_image(int p, const std::vector<double>& blob, std::vector<unsigned char>& img);

}  // namespace ldg
