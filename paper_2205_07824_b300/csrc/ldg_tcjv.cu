// Euler J.v with the element contractions on the tensor cores (tcgen05), affine
// quadrilaterals of order p = 1..4 with p + 2 Gauss points per direction.
//
// The LDG residual of Eq. 1b has three dense linear maps per element, batched over
// elements: interpolation of the nodal state to the volume and face points, the weak
// volume integral against the basis derivatives, and the lift of the face fluxes back
// to the nodes (plus the mass matrix of the BDF time term). Written as matrices over
// all nodes and points of an element (not sum-factorised), each is a GEMM with the
// elements' (element, component) pairs as its 128 rows:
//   interpolation  [128 x NPE] . [NPE x NQV]   (u and the direction v; own face traces
//                  [128 x NPE] . [NPE x 4 NQ];  neighbour traces from the gathered
//                  neighbour face nodes [128 x 4 N1] . [4 N1 x 4 NQ])
//   integration    [128 x 2 NQV] . [2 NQV x NPE]  (both reference derivatives at once)
//   lift           [128 x 4 NQ] . [4 NQ x NPE]
//   mass           [128 x NPE] . [NPE x NPE]
// One CTA owns 32 elements (128 rows). Operands are BF16 in shared memory in the
// 128-byte-swizzle K-major layout; one thread issues tcgen05.mma into FP32 accumulators
// in tensor memory. PASSES = 3 splits every operand x into hi = bf16(x) and
// lo = bf16(x - hi) and forms A B as A_hi B_hi + A_lo B_hi + A_hi B_lo (about 1e-5
// relative: FP32-class contractions from BF16 products); PASSES = 1 keeps A_hi B_hi
// (BF16 contractions, about 1e-2). The pointwise work (the Euler flux and the local
// Lax-Friedrichs flux, both with their tangent along v as dual numbers) is FP32 on
// the CUDA cores between the two MMA phases, reading the accumulators back with
// tcgen05.ld and writing the next phase's operands. The output J.v is FP64 in memory.
//
// Every mbarrier wait is bounded (about a second of SM clock). On a timeout the CTA
// records *err, waits once more (bounded) for its MMAs, writes NaN into its outputs,
// frees its tensor memory and returns, so the caller's Krylov iteration stops on a
// non-finite vector instead of using a wrong one.
#include <cuda_bf16.h>

#include <cstring>
#include <string>
#include <vector>

#include "ldg_kernels.cuh"
#include "ldg_launch.cuh"
#include "ldg_tcgen05.cuh"

namespace ldg {
namespace {

__host__ __device__ constexpr int r16(int x) { return (x + 15) & ~15; }
__host__ __device__ constexpr int r64(int x) { return (x + 63) & ~63; }
// bytes of a K-major BF16 operand of `rows` rows and K columns (64 columns per slab)
__host__ __device__ constexpr int op_bytes(int rows, int K) { return (r64(K) / 64) * rows * 128; }
// byte offset of element (r, k) of such an operand in the 128-byte-swizzle layout:
// slab k / 64; 8-row groups 1024 bytes apart; 16-byte chunk (k / 8) % 8 of row r stored
// at chunk position ((k / 8) % 8) xor (r % 8) (the buffer starts 1024-byte aligned)
__host__ __device__ inline uint32_t sw_off(int rows, int r, int k) {
  return (uint32_t)((k >> 6) * rows * 128 + (r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) & 7) ^ (r & 7)) << 4) +
                    (k & 7) * 2);
}

template <int P, int TH = 256> struct TcShape {
  static constexpr int N1 = P + 1, NQ = P + 2, NPE = N1 * N1, NQV = NQ * NQ, NFP = 4 * NQ;
  // padded GEMM extents (multiples of 16): nodes, volume points, face points, face nodes
  static constexpr int KN = r16(NPE), NV = r16(NQV), NFPp = r16(NFP), KF = r16(4 * N1), NN = KN;
  static constexpr int EPC = 32, ROWS = 128, THREADS = TH;
  // constant operands, rows x K with the hi part in the first K / 2 columns and the lo
  // part in the second (host-built images, concatenated in this order)
  static constexpr int B_BV = op_bytes(NV, 2 * KN), B_BF = op_bytes(NFPp, 2 * KN), B_BN = op_bytes(NFPp, 2 * KF),
                       B_BM = op_bytes(NN, 2 * KN), B_BI = op_bytes(NN, 4 * NV), B_BL = op_bytes(NN, 2 * NFPp);
  static constexpr int O_BV = 0, O_BF = O_BV + B_BV, O_BN = O_BF + B_BF, O_BM = O_BN + B_BN, O_BI = O_BM + B_BM,
                       O_BL = O_BI + B_BI, B_CONST = O_BL + B_BL;
  // per-CTA operands: X = [u_hi | u_lo | v_hi | v_lo] over the nodes, N = the same over
  // the gathered neighbour face nodes, G = [G_hi | G_lo] over (derivative, volume point),
  // H = [H_hi | H_lo] over the face points
  static constexpr int B_X = op_bytes(ROWS, 4 * KN), B_N = op_bytes(ROWS, 4 * KF), B_G = op_bytes(ROWS, 4 * NV),
                       B_H = op_bytes(ROWS, 2 * NFPp);
  // G reuses X and N once the first MMA phase has completed (the pointwise phase reads
  // the interpolated values straight from tensor memory)
  static constexpr int B_T = B_X + B_N;
  static_assert(B_G <= B_T, "G in the X / N region");
  static constexpr int S_CONST = 0, S_T = B_CONST, S_G = S_T, S_H = S_T + B_T, S_GEO = S_H + B_H;
  // per element: Jinv[k][d] (4), detJ, then per face the unit normal and sJ (12), padded
  static constexpr int GEOF = 20;
  // per warp: a transpose tile [8 elements][8 points][16 fields] (row stride padded to
  // 132 floats: the stores of one point are conflict-free and 16-byte aligned)
  static constexpr int WSTR = 132, B_W = 8 * WSTR * 4;
  static constexpr int S_W = S_GEO + EPC * GEOF * 4;
  static constexpr int S_END = S_W + (THREADS / 32) * B_W;
  // tensor-memory columns (FP32 accumulators, one column per GEMM column)
  static constexpr int T_U = 0, T_V = NV, T_FU = 2 * NV, T_FV = T_FU + NFPp, T_NU = T_FV + NFPp,
                       T_NV = T_NU + NFPp, T_M = T_NV + NFPp, T_END = T_M + NN;
  static constexpr int T_R = 0;   // the residual accumulator reuses u's columns (read out by then)
  static constexpr uint32_t T_COLS = T_END <= 32 ? 32 : T_END <= 64 ? 64 : T_END <= 128 ? 128 : 256;
  static_assert(T_END <= 256, "tensor memory");
  // CTAs per SM: at most as many as the 512 tensor-memory columns hold, so that no
  // allocation waits; the dynamic shared memory is padded to enforce it (228 KB per SM,
  // about 4 KB per CTA reserved and static)
  static constexpr int MAXC = 512 / (int)T_COLS;
  static constexpr int SMEM_RAW = S_END + 1024;   // + alignment slack of the dynamic buffer
  static constexpr int SMEM_CAP = (228 * 1024) / (MAXC + 1) - 3 * 1024;
  static constexpr int SMEM = SMEM_RAW > SMEM_CAP ? SMEM_RAW : SMEM_CAP;
  static constexpr int MINB = TH == 256 && SMEM <= 110 * 1024 ? 2 : 1;   // register budget for 2 CTAs per SM
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// hi / lo BF16 parts of x at column k (hi) and k + lo_off (lo)
template <int PASSES> __device__ __forceinline__ void put_split(unsigned char* buf, int rows, int r, int k, int lo_off,
                                                                float x) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(x);
  *(__nv_bfloat16*)(buf + sw_off(rows, r, k)) = hi;
  if constexpr (PASSES == 3) *(__nv_bfloat16*)(buf + sw_off(rows, r, k + lo_off)) = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Eight consecutive operand values (columns col .. col + 7 of row r, col a multiple of 8:
// one 16-byte chunk of the swizzled layout) as BF16 hi parts, and for PASSES = 3 the lo
// parts at col + lo_off, each with one 16-byte store.
template <int PASSES>
__device__ __forceinline__ void put8(unsigned char* buf, int rows, int r, int col, int lo_off, const float* x) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * t], x[2 * t + 1]);
    h[t] = *reinterpret_cast<const uint32_t*>(&hb);
    if constexpr (PASSES == 3) {
      const float2 hf = __bfloat1622float2(hb);
      const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * t] - hf.x, x[2 * t + 1] - hf.y);
      l[t] = *reinterpret_cast<const uint32_t*>(&lb);
    }
  }
  *reinterpret_cast<uint4*>(buf + sw_off(rows, r, col)) = make_uint4(h[0], h[1], h[2], h[3]);
  if constexpr (PASSES == 3)
    *reinterpret_cast<uint4*>(buf + sw_off(rows, r, col + lo_off)) = make_uint4(l[0], l[1], l[2], l[3]);
}

// descriptor of the 16 K-columns of an operand starting at column k (k a multiple of 16)
__device__ __forceinline__ uint64_t kdesc(const unsigned char* op, int rows, int k) {
  return sw128_desc(op + (k >> 6) * rows * 128 + (k & 63) * 2);
}

// D[128][N] (+)= A[:, ka .. ka + K) B[:, kb .. kb + K)^T, the lo parts at +alo / +blo
template <int PASSES>
__device__ __forceinline__ void mma_split(uint32_t d, const unsigned char* A, int ka, int alo, const unsigned char* B,
                                          int brows, int kb, int blo, int K, int N, bool acc) {
  const uint32_t idesc = bf16_idesc(128, N);
  int on = acc ? 1 : 0;
  for (int s = 0; s < K; s += 16) {
    tc_mma(d, kdesc(A, 128, ka + s), kdesc(B, brows, kb + s), idesc, on);
    on = 1;
    if constexpr (PASSES == 3) {
      tc_mma(d, kdesc(A, 128, ka + alo + s), kdesc(B, brows, kb + s), idesc, 1);
      tc_mma(d, kdesc(A, 128, ka + s), kdesc(B, brows, kb + blo + s), idesc, 1);
    }
  }
}


template <int P, int PASSES, int TH>
__global__ void __launch_bounds__(TH, TcShape<P, TH>::MINB) k_euler_jv_tc(KArgs a, const unsigned char* __restrict__ cimg, int* err) {
  typedef TcShape<P, TH> T;
  typedef TensorEl<2, P, P + 2> EL;
  typedef Dual<float> S;
  constexpr int GEO = Geo<2>::FACE + 4 * 3;   // doubles per element record
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(1024) unsigned char tcj_raw[];
  // the swizzle is a function of the shared-memory address: align the operands to 1024
  unsigned char* sm = tcj_raw + ((1024u - (smem_u32(tcj_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bar_a, bar_d;
  __shared__ uint32_t tmem_base;
  __shared__ int ok_s;
  __shared__ MPar<float> MPs[T::EPC];
  __shared__ int s_nb[T::EPC * 4], s_nbase[T::EPC * 4], s_nstep[T::EPC * 4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int e0 = blockIdx.x * T::EPC;
  const int ne = min(T::EPC, a.E - e0);
  if (!cta_active(a, e0, ne)) return;

  unsigned char* sC = sm + T::S_CONST;
  unsigned char* sX = sm + T::S_T;
  unsigned char* sN = sm + T::S_T + T::B_X;
  unsigned char* sG = sm + T::S_G;
  unsigned char* sH = sm + T::S_H;
  float* gs = (float*)(sm + T::S_GEO);
  const double* u = (const double*)a.u;
  const double* v = (const double*)a.v;
  const float* W = a.opsf + EL::OW;   // 1-D Gauss weights

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(T::T_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar_a, 1);
    mbar_init(&bar_d, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ok_s = 1;
  }
  // ---- phase 0: constant operands, geometry, the element and neighbour operands
  {
    const uint4* src = (const uint4*)cimg;
    uint4* dst = (uint4*)sC;
    for (int i = tid; i < T::B_CONST / 16; i += T::THREADS) dst[i] = src[i];
  }
  for (int i = tid; i < T::EPC * T::GEOF; i += T::THREADS) {
    const int e = i / T::GEOF, j = i % T::GEOF;
    float x = 0.f;
    if (e < ne) {
      const double* g = a.geo + (size_t)(e0 + e) * GEO;
      if (j < 5) x = (float)g[j];                                    // Jinv, detJ
      else if (j < 17) x = (float)g[Geo<2>::FACE + (j - 5)];         // face f: n0, n1, sJ at 5 + 3 f
    }
    gs[i] = x;
  }
  for (int e = tid; e < T::EPC; e += T::THREADS) MPs[e] = mpar<float>(e < ne ? elem_mp(a, e0 + e) : a.mp);
  // per (element, face): the neighbour (or -1 / -2), and its face-node run in this
  // element's face-node order, node = base + j * step (a reversed edge reverses the run:
  // the Gauss-Lobatto nodes and the Gauss points are symmetric)
  for (int t = tid; t < T::EPC * 4; t += T::THREADS) {
    const int e = t >> 2, f = t & 3;
    int nb = -1, base = 0, step = 0;
    if (e < ne) {
      nb = a.nbr[(size_t)(e0 + e) * 4 + f];
      if (nb >= 0) {
        const int code = a.nbf[(size_t)(e0 + e) * 4 + f];
        const bool rev = a.perm[(code >> 3) * T::NQ] != 0;
        const int n0 = EL::face_node(code & 7, 0), n1 = EL::face_node(code & 7, T::N1 - 1);
        const int st = (n1 - n0) / (T::N1 - 1);
        base = rev ? n1 : n0;
        step = rev ? -st : st;
      }
    }
    s_nb[t] = nb;
    s_nbase[t] = base;
    s_nstep[t] = step;
  }
  __syncthreads();   // the face runs
  // the element's state and the neighbours' face nodes: every load of a thread is
  // issued before its conversions and stores
  {
    constexpr int IS = T::ROWS * T::KN / T::THREADS, IG = T::ROWS * T::KF / T::THREADS;
    static_assert(T::ROWS * T::KN % T::THREADS == 0 && T::ROWS * T::KF % T::THREADS == 0, "operand tiles");
    float su[IS], sv[IS], gu[IG], gv[IG];
#pragma unroll
    for (int j = 0; j < IS; ++j) {
      const int i = tid + j * T::THREADS, r = i / T::KN, n = i % T::KN, e = r >> 2;
      su[j] = sv[j] = 0.f;
      if (e < ne && n < T::NPE) {
        const size_t gi = ((size_t)e0 * 4 + r) * T::NPE + n;
        su[j] = (float)__ldg(u + gi);
        sv[j] = (float)__ldg(v + gi);
      }
    }
#pragma unroll
    for (int j = 0; j < IG; ++j) {
      const int i = tid + j * T::THREADS, r = i / T::KF, k = i % T::KF, e = r >> 2, c = r & 3;
      gu[j] = gv[j] = 0.f;
      if (k < 4 * T::N1) {
        const int f = k / T::N1, jj = k % T::N1, t = e * 4 + f;
        const int nb = s_nb[t];
        if (nb >= 0) {
          const size_t gi = ((size_t)nb * 4 + c) * T::NPE + s_nbase[t] + jj * s_nstep[t];
          gu[j] = (float)__ldg(u + gi);
          gv[j] = (float)__ldg(v + gi);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < IS; ++j) {
      const int i = tid + j * T::THREADS, r = i / T::KN, n = i % T::KN;
      put_split<PASSES>(sX, T::ROWS, r, n, T::KN, su[j]);
      put_split<PASSES>(sX, T::ROWS, r, 2 * T::KN + n, T::KN, sv[j]);
    }
#pragma unroll
    for (int j = 0; j < IG; ++j) {
      const int i = tid + j * T::THREADS, r = i / T::KF, k = i % T::KF;
      put_split<PASSES>(sN, T::ROWS, r, k, T::KF, gu[j]);
      put_split<PASSES>(sN, T::ROWS, r, 2 * T::KF + k, T::KF, gv[j]);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  // ---- phase A MMAs: interpolation to the volume points, own and neighbour face
  // traces, and the reference mass matrix applied to v
  if (tid == 0) {
    mma_split<PASSES>(tmem + T::T_U, sX, 0, T::KN, sC + T::O_BV, T::NV, 0, T::KN, T::KN, T::NV, false);
    mma_split<PASSES>(tmem + T::T_V, sX, 2 * T::KN, T::KN, sC + T::O_BV, T::NV, 0, T::KN, T::KN, T::NV, false);
    mma_split<PASSES>(tmem + T::T_FU, sX, 0, T::KN, sC + T::O_BF, T::NFPp, 0, T::KN, T::KN, T::NFPp, false);
    mma_split<PASSES>(tmem + T::T_FV, sX, 2 * T::KN, T::KN, sC + T::O_BF, T::NFPp, 0, T::KN, T::KN, T::NFPp, false);
    mma_split<PASSES>(tmem + T::T_NU, sN, 0, T::KF, sC + T::O_BN, T::NFPp, 0, T::KF, T::KF, T::NFPp, false);
    mma_split<PASSES>(tmem + T::T_NV, sN, 2 * T::KF, T::KF, sC + T::O_BN, T::NFPp, 0, T::KF, T::KF, T::NFPp, false);
    mma_split<PASSES>(tmem + T::T_M, sX, 2 * T::KN, T::KN, sC + T::O_BM, T::NN, 0, T::KN, T::KN, T::NN, false);
    tc_commit(&bar_a);
  }
  {
    const bool okw = __all_sync(0xffffffffu, mbar_wait(&bar_a, 0));
    if (!okw) {
      if (lane == 0) atomicExch(err, 1);
      ok_s = 0;
      (void)mbar_wait(&bar_a, 0);   // a second bounded wait: the MMAs may still be running
    }
  }
  __syncthreads();
  const bool ok_a = ok_s != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");

  // ---- phase C: pointwise fluxes with their tangents; the integration operand G (over
  // the X / N region, free now) and the lift operand H. Warp w reads tensor-memory lanes
  // 32 (w % 4) .. + 32, i.e. rows (e, c) of 8 elements; the 16-column chunks of the volume
  // and face points alternate between the warps w and w + 4. Eight points at a time go
  // through the warp's transpose tile, after which lane (e, c) holds all components at
  // the points c and c + 4 of the eight.
  if (ok_a) {
    const int quarter = warp & 3, group = warp >> 2;
    constexpr int NGROUPS = T::THREADS / 128;
    const int c = lane & 3, el = lane >> 2, e = quarter * 8 + el;
    const uint32_t lrow = tmem + ((uint32_t)(quarter * 32) << 16);
    constexpr int NVC = T::NV / 16, NFC = T::NFPp / 16;
    float* wt = (float*)(sm + T::S_W) + warp * (T::B_W / 4) + el * T::WSTR;
    const bool live = e < ne;
    const float* ge = gs + e * T::GEOF;
    for (int ch = group; ch < NVC + NFC; ch += NGROUPS) {   // warp-uniform
      if (ch < NVC) {
        const int q0 = ch * 16;
        float U[16], V[16];
        tc_ld16(lrow + (uint32_t)(T::T_U + q0), U);
        tc_ld16(lrow + (uint32_t)(T::T_V + q0), V);
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            wt[i * 16 + c] = U[hc * 8 + i];
            wt[i * 16 + 4 + c] = V[hc * 8 + i];
          }
          __syncwarp();
          float g2[2][8];
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {
            const int i = c + 4 * jj, q = q0 + hc * 8 + i;
            const float4 uu = *(const float4*)(wt + i * 16), vv = *(const float4*)(wt + i * 16 + 4);
#pragma unroll
            for (int j = 0; j < 8; ++j) g2[jj][j] = 0.f;
            if (live && q < T::NQV) {
              const S st[4] = {S(uu.x, vv.x), S(uu.y, vv.y), S(uu.z, vv.z), S(uu.w, vv.w)};
              S f[8];
              EulerModel::flux(st, (const S*)nullptr, f, MPs[e]);
              const float wq = W[q % T::NQ] * W[q / T::NQ] * ge[4];
#pragma unroll
              for (int cc = 0; cc < 4; ++cc)
#pragma unroll
                for (int k = 0; k < 2; ++k)
                  g2[jj][cc * 2 + k] = -wq * (f[cc * 2].d * ge[k * 2] + f[cc * 2 + 1].d * ge[k * 2 + 1]);
            }
          }
          __syncwarp();
          // G_{cc,k} at the 8 points of the element through the tile, then one 16-byte
          // store per (row, derivative) segment: lane (e, c) packs j = c and c + 4
#pragma unroll
          for (int jj = 0; jj < 2; ++jj)
#pragma unroll
            for (int j = 0; j < 8; ++j) wt[(c + 4 * jj) * 16 + j] = g2[jj][j];
          __syncwarp();
#pragma unroll
          for (int sg = 0; sg < 2; ++sg) {
            const int j = c + 4 * sg, cc = j >> 1, k = j & 1;
            float x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = wt[i * 16 + j];
            put8<PASSES>(sG, T::ROWS, e * 4 + cc, k * T::NV + q0 + hc * 8, 2 * T::NV, x);
          }
          __syncwarp();
        }
      } else {
        const int p0 = (ch - NVC) * 16;
        float FU[16], FV[16], NU[16], NVv[16];
        tc_ld16(lrow + (uint32_t)(T::T_FU + p0), FU);
        tc_ld16(lrow + (uint32_t)(T::T_FV + p0), FV);
        tc_ld16(lrow + (uint32_t)(T::T_NU + p0), NU);
        tc_ld16(lrow + (uint32_t)(T::T_NV + p0), NVv);
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            wt[i * 16 + c] = FU[hc * 8 + i];
            wt[i * 16 + 4 + c] = FV[hc * 8 + i];
            wt[i * 16 + 8 + c] = NU[hc * 8 + i];
            wt[i * 16 + 12 + c] = NVv[hc * 8 + i];
          }
          __syncwarp();
          float h2[2][4];
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {
            const int i = c + 4 * jj, pt = p0 + hc * 8 + i;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) h2[jj][cc] = 0.f;
            if (live && pt < T::NFP) {
              const float4 um_ = *(const float4*)(wt + i * 16), vm_ = *(const float4*)(wt + i * 16 + 4);
              const int f = pt / T::NQ, k = pt % T::NQ;
              const S um[4] = {S(um_.x, vm_.x), S(um_.y, vm_.y), S(um_.z, vm_.z), S(um_.w, vm_.w)};
              const float* gf = ge + 5 + 3 * f;
              const float nrm[2] = {gf[0], gf[1]};
              const float w = W[k] * gf[2];
              const int nb = s_nb[e * 4 + f];
              S fh[4];
              if (nb >= 0) {
                const float4 up_ = *(const float4*)(wt + i * 16 + 8), vp_ = *(const float4*)(wt + i * 16 + 12);
                const S up[4] = {S(up_.x, vp_.x), S(up_.y, vp_.y), S(up_.z, vp_.z), S(up_.w, vp_.w)};
                EulerModel::fhat(um, up, (const S*)nullptr, (const S*)nullptr, nrm, fh, MPs[e]);
              } else if (nb == -2) {
                EulerModel::fhat_wall(um, (const S*)nullptr, nrm, fh, MPs[e]);
              } else {
                // far field: the exact state (no tangent) at the face point
                double xi[2], x[3], gd[4] = {0.0, 0.0, 0.0, 0.0};
                face_xi<EL>(a.ops, f, k, xi);
                phys_x<2>(a.geo + (size_t)(e0 + e) * GEO, xi, x);
                exact_state<2>(elem_mp(a, e0 + e), 4, x, a.t_dev ? *a.t_dev : a.t, gd);
                const float gb[4] = {(float)gd[0], (float)gd[1], (float)gd[2], (float)gd[3]};
                EulerModel::fhat_bnd(um, (const S*)nullptr, gb, nrm, fh, MPs[e]);
              }
#pragma unroll
              for (int cc = 0; cc < 4; ++cc) h2[jj][cc] = fh[cc].d * w;
            }
          }
          __syncwarp();
#pragma unroll
          for (int jj = 0; jj < 2; ++jj)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) wt[(c + 4 * jj) * 16 + cc] = h2[jj][cc];
          __syncwarp();
          {
            float x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = wt[i * 16 + c];
            put8<PASSES>(sH, T::ROWS, e * 4 + c, p0 + hc * 8, T::NFPp, x);
          }
          __syncwarp();
        }
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // ---- phase D MMAs: volume integration and face lift into one accumulator
  if (ok_a && tid == 0) {
    mma_split<PASSES>(tmem + T::T_R, sG, 0, 2 * T::NV, sC + T::O_BI, T::NN, 0, 2 * T::NV, 2 * T::NV, T::NN, false);
    mma_split<PASSES>(tmem + T::T_R, sH, 0, T::NFPp, sC + T::O_BL, T::NN, 0, T::NFPp, T::NFPp, T::NN, true);
    tc_commit(&bar_d);
  }
  if (ok_a) {
    const bool okw = __all_sync(0xffffffffu, mbar_wait(&bar_d, 0));
    if (!okw) {
      if (lane == 0) atomicExch(err, 1);
      ok_s = 0;
      (void)mbar_wait(&bar_d, 0);
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // ---- phase E: J.v = integration + lift + a0/dt detJ (M_ref v), staged in shared
  // memory (G is free once the second MMA phase has completed) and stored coalesced
  constexpr int OS = T::NPE + 1;   // padded row stride (doubles) of the staging buffer
  static_assert(T::ROWS * OS * 8 <= T::B_G, "output staging");
  double* sO = (double*)sG;
  const bool ok = ok_s != 0;
  if (warp < 4 && ok) {
    const int r = warp * 32 + lane, e = r >> 2;
    const uint32_t lrow = tmem + ((uint32_t)(warp * 32) << 16);
    const float mt = (float)a.a0dt * gs[e * T::GEOF + 4];
    for (int c0 = 0; c0 < T::NN; c0 += 16) {
      float rv[16], mv[16];
      tc_ld16(lrow + (uint32_t)(T::T_R + c0), rv);
      if (a.a0dt != 0.0) tc_ld16(lrow + (uint32_t)(T::T_M + c0), mv);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (c0 + i < T::NPE) sO[r * OS + c0 + i] = (double)rv[i] + (a.a0dt != 0.0 ? (double)(mt * mv[i]) : 0.0);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  {
    double* out = (double*)a.out + (size_t)e0 * 4 * T::NPE;
    for (int i = tid; i < ne * 4 * T::NPE; i += T::THREADS) out[i] = ok ? sO[(i / T::NPE) * OS + i % T::NPE] : nan("");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T::T_COLS) : "memory");
  }
}

// 1-D Lagrange basis of the Gauss-Lobatto nodes at the face end points: delta
inline double lend(int j, int n1, int side) { return j == (side ? n1 - 1 : 0) ? 1.0 : 0.0; }

inline uint16_t bf16_bits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);   // round to nearest even (finite values)
  return (uint16_t)(u >> 16);
}
inline float bf16_val(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}

template <int P> void build_image(const std::vector<double>& blob, std::vector<unsigned char>& img) {
  typedef TcShape<P> T;
  const int N1 = T::N1, NQ = T::NQ;
  const double* B1 = blob.data();               // B[NQ][N1] basis at the Gauss points
  const double* D1 = B1 + NQ * N1;              // D[NQ][N1] its derivative
  const double* W = D1 + NQ * N1;               // Gauss weights
  img.assign(T::B_CONST, 0);
  // hi part at column k, lo part at column k + lo (both BF16 bits)
  auto put = [&](int off, int rows, int r, int k, int lo, double x) {
    const uint16_t h = bf16_bits((float)x);
    const uint16_t l = bf16_bits((float)(x - (double)bf16_val(h)));
    std::memcpy(&img[off + sw_off(rows, r, k)], &h, 2);
    std::memcpy(&img[off + sw_off(rows, r, k + lo)], &l, 2);
  };
  // value of node n (i0 + N1 i1) at face point (f, k) of face f = 2 axis + side
  auto face_val = [&](int n, int f, int k) {
    const int i0 = n % N1, i1 = n / N1, ax = f >> 1, side = f & 1;
    return ax == 0 ? lend(i0, N1, side) * B1[k * N1 + i1] : B1[k * N1 + i0] * lend(i1, N1, side);
  };
  for (int q = 0; q < T::NQV; ++q)
    for (int n = 0; n < T::NPE; ++n) {
      const int q0 = q % NQ, q1 = q / NQ, i0 = n % N1, i1 = n / N1;
      put(T::O_BV, T::NV, q, n, T::KN, B1[q0 * N1 + i0] * B1[q1 * N1 + i1]);
      put(T::O_BI, T::NN, n, q, 2 * T::NV, D1[q0 * N1 + i0] * B1[q1 * N1 + i1]);
      put(T::O_BI, T::NN, n, T::NV + q, 2 * T::NV, B1[q0 * N1 + i0] * D1[q1 * N1 + i1]);
    }
  for (int f = 0; f < 4; ++f)
    for (int k = 0; k < NQ; ++k) {
      const int pt = f * NQ + k;
      for (int n = 0; n < T::NPE; ++n) {
        put(T::O_BF, T::NFPp, pt, n, T::KN, face_val(n, f, k));
        put(T::O_BL, T::NN, n, pt, T::NFPp, face_val(n, f, k));
      }
      for (int j = 0; j < N1; ++j) put(T::O_BN, T::NFPp, pt, f * N1 + j, T::KF, B1[k * N1 + j]);
    }
  for (int n = 0; n < T::NPE; ++n)
    for (int m = 0; m < T::NPE; ++m) {
      double s = 0.0;
      for (int q1 = 0; q1 < NQ; ++q1)
        for (int q0 = 0; q0 < NQ; ++q0)
          s += W[q0] * W[q1] * B1[q0 * N1 + n % N1] * B1[q1 * N1 + n / N1] * B1[q0 * N1 + m % N1] *
               B1[q1 * N1 + m / N1];
      put(T::O_BM, T::NN, n, m, T::KN, s);
    }
}

template <int P, int PASSES, int TH> cudaError_t launch_th(const KArgs& a, const unsigned char* img, int* err, unsigned grid,
                                                          cudaStream_t s) {
  typedef TcShape<P, TH> T;
  static const cudaError_t attr = cudaFuncSetAttribute(k_euler_jv_tc<P, PASSES, TH>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
  if (attr != cudaSuccess) return attr;
  k_euler_jv_tc<P, PASSES, TH><<<grid, TH, T::SMEM, s>>>(a, img, err);
  return cudaGetLastError();
}

// A grid of at most two CTAs per SM runs one 512-thread CTA per SM; larger grids run
// 256-thread CTAs, two per SM where shared memory and tensor memory allow.
template <int P, int PASSES> cudaError_t launch(const KArgs& a, const unsigned char* img, int* err, cudaStream_t s) {
  static const int n_sm = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 148;
    return n;
  }();
  if (a.E <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((a.E + 31) / 32);
  return (int)grid <= 2 * n_sm ? launch_th<P, PASSES, 512>(a, img, err, grid, s) : launch_th<P, PASSES, 256>(a, img, err, grid, s);
}

template <int P> cudaError_t launch_p(const KArgs& a, const unsigned char* img, int passes, int* err, cudaStream_t s) {
  return passes == 3 ? launch<P, 3>(a, img, err, s) : launch<P, 1>(a, img, err, s);
}

}  // namespace

TcJvFn tcjv_launcher(int p) {
  switch (p) {
    case 1: return launch_p<1>;
    case 2: return launch_p<2>;
    case 3: return launch_p<3>;
    case 4: return launch_p<4>;
    default: return nullptr;
  }
}

bool build_tcjv_image(int p, const std::vector<double>& blob, std::vector<unsigned char>& img) {
  switch (p) {
    case 1: build_image<1>(blob, img); return true;
    case 2: build_image<2>(blob, img); return true;
    case 3: build_image<3>(blob, img); return true;
    case 4: build_image<4>(blob, img); return true;
    default: return false;
  }
}

}  // namespace ldg
