// FP32 propagation of a batch of states through a chain of propagators for
// n > 81 (Alg. 2 applied to every state, Sec. 3.2), in the reduced form
//   R_{t+1} = c_t (R_t + R_t D_t^T),   D_t = P_t - I,
// where c_t = 1 / Tr(R_t) when the trace is renormalised (deferred by one
// step: the trace of R_t is read at the start of step t + 1 and applied in its
// epilogue, which is the same state up to rounding) and c_t = 1 otherwise.
//
// Layout ("planes", FP32, K-major so that tiles stream with 16-byte async
// copies and no transposition in the loop):
//   D^T of every slice   Dt[s][2][Kp][Np]  planes Re, Im, (k, j)
//   states               Rt[2][Kp][Bp]     planes Re, Im, (k, b)
// Kp = n rounded up to 16, Np = n rounded up to 64, Bp = B rounded up to 64;
// padding rows and columns hold zeros (the step keeps them zero).
//
// The step is a complex GEMM  O[b][j] = sum_k R[b][k] D[j][k]  in Gauss's
// three-real-product form (t1 = Re Re, t2 = Im Im, t3 = (Re+Im)(Re+Im);
// Re = t1 - t2, Im = t3 - t1 - t2; the operand sums are formed in registers,
// which keeps shared-memory traffic at two planes): 64 x 64 output tiles, 256 threads with
// 4 x 4 complex outputs each (fragments double-buffered in registers), a
// four-stage cp.async ring of 16-deep K blocks, two CTAs per SM.  When there
// are fewer tiles than two per SM the K range is split over CTAs.  If the
// split CTAs of a tile fit on the GPU as one thread-block cluster, each keeps
// its partial tile in shared memory and, after a cluster barrier, sums one
// share of the tile's rows over all partials through distributed shared
// memory; otherwise each writes its partial to global scratch and the CTA
// that takes the last ticket (atomic, no waiting) sums them.  Either way the
// partials are added in split order, so the result does not depend on
// arrival order.  A chain of at least two steps whose split CTAs form
// clusters runs as one persistent launch (chain32_persist_kernel below).
#include "lb_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>

namespace lb {

namespace {

constexpr int CB = 64;        // tile rows (states) and columns (outputs)
constexpr int CK = 16;        // K per stage
constexpr int CSTAGE = 4;     // cp.async ring depth
constexpr int kChainTM = 4;  // complex outputs per thread along the states (TM = 8 measured 27% slower)
constexpr int NPL = 2;                         // planes per operand (Re, Im)
constexpr int OPER_FLOATS = NPL * CK * CB;     // one operand
constexpr int STAGE_FLOATS = 2 * OPER_FLOATS;  // A (states) and B (D^T)
constexpr size_t STEP_SMEM = (size_t)CSTAGE * STAGE_FLOATS * sizeof(float);

struct ChainDims {
  int n, d, B, Kp, Np, Bp;
};

__device__ __forceinline__ void cp16(float* s, const float* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Programmatic dependent launch: a step launched with programmatic stream
// serialisation may start while the previous step drains; it reads nothing
// the previous step writes before griddep_wait() (a no-op otherwise).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// Output of four consecutive states b..b+3 at output index j: add the
// residual R[b][j], multiply by the per-state factor, store both planes.
__device__ __forceinline__ void chain_finish(const ChainDims& g, const float* __restrict__ Rt,
                                             float* __restrict__ Ot, const float2* cs, int j, int b, float4 ar,
                                             float4 ai) {
  if (j >= g.Kp) return;
  const long long pl = (long long)g.Kp * g.Bp;
  const long long idx = (long long)j * g.Bp + b;
  const float4 rr = f4add(ar, *(const float4*)(Rt + idx));
  const float4 ri = f4add(ai, *(const float4*)(Rt + pl + idx));
  const float vr[4] = {rr.x, rr.y, rr.z, rr.w}, vi[4] = {ri.x, ri.y, ri.z, ri.w};
  float orr[4], oii[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const float2 c = cs[e];
    orr[e] = vr[e] * c.x - vi[e] * c.y;
    oii[e] = vr[e] * c.y + vi[e] * c.x;
  }
  *(float4*)(Ot + idx) = make_float4(orr[0], orr[1], orr[2], orr[3]);
  *(float4*)(Ot + pl + idx) = make_float4(oii[0], oii[1], oii[2], oii[3]);
}

// TM states x 4 outputs per thread: TM = 4 with 256 threads (2 x 4 warps
// of 8 x 4 threads) or TM = 8 with 128 threads (2 x 2 warps of 4 x 8).
template <bool RENORM, int TM>
__global__ void __launch_bounds__(1024 / TM, 2)
    chain32_step_kernel(ChainDims g, int kps, const float* __restrict__ Dt, const float* __restrict__ Rt,
                        float* __restrict__ Ot, float* __restrict__ part, unsigned* __restrict__ cnt,
                        int use_cluster) {
  constexpr int NT = 1024 / TM;  // threads
  constexpr int NQ = NT / CB;    // partial trace sums per state
  extern __shared__ __align__(16) float sm[];
  __shared__ float2 cs[CB];
  __shared__ float2 trp[NQ][CB];
  __shared__ int is_last;
  const int tid = threadIdx.x;
  const int j0 = blockIdx.x * CB, m0 = blockIdx.y * CB, z = blockIdx.z, splits = gridDim.z;
  const int kt0 = z * kps;
  const int kt1 = min(g.Kp / CK, kt0 + kps);
  const int nkt = kt1 - kt0;
  const long long pA = (long long)g.Kp * g.Bp, pB = (long long)g.Kp * g.Np;

  auto loadA = [&](int stage, int kt) {  // states: written by the previous step
    float* sA = sm + stage * STAGE_FLOATS;
    const int k0 = kt * CK;
    for (int c = tid; c < NPL * CK * (CB / 4); c += NT) {
      const int p = c / (CK * (CB / 4)), r = (c / (CB / 4)) % CK, q = c % (CB / 4);
      cp16(sA + (p * CK + r) * CB + 4 * q, Rt + p * pA + (long long)(k0 + r) * g.Bp + m0 + 4 * q);
    }
  };
  auto loadB = [&](int stage, int kt) {  // D^T: written before the chain started
    float* sB = sm + stage * STAGE_FLOATS + OPER_FLOATS;
    const int k0 = kt * CK;
    for (int c = tid; c < NPL * CK * (CB / 4); c += NT) {
      const int p = c / (CK * (CB / 4)), r = (c / (CB / 4)) % CK, q = c % (CB / 4);
      cp16(sB + (p * CK + r) * CB + 4 * q, Dt + p * pB + (long long)(k0 + r) * g.Np + j0 + 4 * q);
    }
  };
  // the first stages of D^T before the wait for the previous step, then the states
#pragma unroll
  for (int s = 0; s < CSTAGE - 1; s++)
    if (s < nkt) loadB(s, kt0 + s);
  griddep_wait();
#pragma unroll
  for (int s = 0; s < CSTAGE - 1; s++) {
    if (s < nkt) loadA(s, kt0 + s);
    cp_commit();
  }
  // per-state factor 1 / Tr(R_b) (complex; 0 for padding states): the d
  // diagonal entries of the CTA's 64 states are loaded by all threads at
  // once (NQ partial sums per state, combined after the K loop), so no
  // warp waits on a chain of dependent loads before its first K block
  if (RENORM) {
    const int b = m0 + (tid & (CB - 1)), q0 = tid / CB;  // q0 in 0..NQ-1
    float tr = 0.f, ti = 0.f;
    if (b < g.B) {
#pragma unroll
      for (int u = 0; u < 32 / NQ; u++) {  // d <= 27 < 32
        const int i = q0 + NQ * u;
        if (i < g.d) {
          const long long k = (long long)i * (g.d + 1) * g.Bp + b;
          tr += __ldg(Rt + k);
          ti += __ldg(Rt + pA + k);
        }
      }
    }
    trp[q0][tid & (CB - 1)] = make_float2(tr, ti);
  }
  const int w = tid >> 5, l = tid & 31;
  // this thread's TM states (am..) and 4 outputs (bn..)
  const int am = TM == 4 ? (w >> 2) * 32 + (l & 7) * 4 : (w >> 1) * 32 + (l & 3) * 8;
  const int bn = TM == 4 ? (w & 3) * 16 + (l >> 3) * 4 : (w & 1) * 32 + (l >> 2) * 4;
  float t1[TM][4], t2[TM][4], t3[TM][4];
#pragma unroll
  for (int i = 0; i < TM; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) t1[i][j] = t2[i][j] = t3[i][j] = 0.f;

  for (int it = 0; it < nkt; it++) {
    cp_wait<CSTAGE - 2>();
    __syncthreads();
    {
      const int nx = it + CSTAGE - 1;
      if (nx < nkt) {
        loadA(nx % CSTAGE, kt0 + nx);
        loadB(nx % CSTAGE, kt0 + nx);
      }
      cp_commit();
    }
    const float* sA = sm + (it % CSTAGE) * STAGE_FLOATS;
    const float* sB = sA + OPER_FLOATS;
    // fragments of step k + 1 are read while step k multiplies
    constexpr int QA = TM / 4;  // float4 per A plane
    float4 fa[2][NPL][QA], fb[2][NPL];
#pragma unroll
    for (int p = 0; p < NPL; p++) {
#pragma unroll
      for (int h = 0; h < QA; h++) fa[0][p][h] = *(const float4*)(sA + (p * CK) * CB + am + 4 * h);
      fb[0][p] = *(const float4*)(sB + (p * CK) * CB + bn);
    }
#pragma unroll
    for (int k = 0; k < CK; k++) {
      const int cur = k & 1;
      if (k + 1 < CK) {
#pragma unroll
        for (int p = 0; p < NPL; p++) {
#pragma unroll
          for (int h = 0; h < QA; h++) fa[cur ^ 1][p][h] = *(const float4*)(sA + (p * CK + k + 1) * CB + am + 4 * h);
          fb[cur ^ 1][p] = *(const float4*)(sB + (p * CK + k + 1) * CB + bn);
        }
      }
      float ar[TM], ai[TM], as[TM];
#pragma unroll
      for (int h = 0; h < QA; h++) {
        ar[4 * h] = fa[cur][0][h].x; ar[4 * h + 1] = fa[cur][0][h].y;
        ar[4 * h + 2] = fa[cur][0][h].z; ar[4 * h + 3] = fa[cur][0][h].w;
        ai[4 * h] = fa[cur][1][h].x; ai[4 * h + 1] = fa[cur][1][h].y;
        ai[4 * h + 2] = fa[cur][1][h].z; ai[4 * h + 3] = fa[cur][1][h].w;
      }
#pragma unroll
      for (int i = 0; i < TM; i++) as[i] = ar[i] + ai[i];
      const float br[4] = {fb[cur][0].x, fb[cur][0].y, fb[cur][0].z, fb[cur][0].w};
      const float bi[4] = {fb[cur][1].x, fb[cur][1].y, fb[cur][1].z, fb[cur][1].w};
      const float bs[4] = {br[0] + bi[0], br[1] + bi[1], br[2] + bi[2], br[3] + bi[3]};
#pragma unroll
      for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          t1[i][j] = fmaf(ar[i], br[j], t1[i][j]);
          t2[i][j] = fmaf(ai[i], bi[j], t2[i][j]);
          t3[i][j] = fmaf(as[i], bs[j], t3[i][j]);
        }
    }
  }
  cp_wait<0>();
  griddep_launch();  // the next step may start its prologue
  __syncthreads();
  if (tid < CB) {
    float2 c = make_float2(0.f, 0.f);
    if (m0 + tid < g.B) {
      if (RENORM) {
        float tr = 0.f, ti = 0.f;
#pragma unroll
        for (int q = 0; q < NQ; q++) {
          tr += trp[q][tid].x;
          ti += trp[q][tid].y;
        }
        const float m2 = tr * tr + ti * ti;
        c = make_float2(tr / m2, -ti / m2);
      } else {
        c = make_float2(1.f, 0.f);
      }
    }
    cs[tid] = c;
  }
  __syncthreads();

  float re[TM][4], im[TM][4];
#pragma unroll
  for (int i = 0; i < TM; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      re[i][j] = t1[i][j] - t2[i][j];
      im[i][j] = t3[i][j] - t1[i][j] - t2[i][j];
    }
  // four consecutive states h*4.. of column j as float4
  auto quad_re = [&](int h, int j) { return make_float4(re[4 * h][j], re[4 * h + 1][j], re[4 * h + 2][j], re[4 * h + 3][j]); };
  auto quad_im = [&](int h, int j) { return make_float4(im[4 * h][j], im[4 * h + 1][j], im[4 * h + 2][j], im[4 * h + 3][j]); };

  if (splits == 1) {
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int h = 0; h < TM / 4; h++)
        chain_finish(g, Rt, Ot, cs + am + 4 * h, j0 + bn + j, m0 + am + 4 * h, quad_re(h, j), quad_im(h, j));
    return;
  }
  if (use_cluster) {
    // partial tile [2][CB (j)][CB (b)] in this CTA's (idle) ring; CTA r of
    // the cluster (r = the K split) finishes rows [r * rows, (r + 1) * rows)
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    float* Ps = sm;
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int h = 0; h < TM / 4; h++) {
        *(float4*)(Ps + (bn + j) * CB + am + 4 * h) = quad_re(h, j);
        *(float4*)(Ps + CB * CB + (bn + j) * CB + am + 4 * h) = quad_im(h, j);
      }
    cl.sync();
    const int rank = (int)cl.block_rank();
    const int rows = (CB + splits - 1) / splits;
    const int jl0 = rank * rows, jl1 = min(CB, jl0 + rows);
    const float* src[8];
#pragma unroll
    for (int zz = 0; zz < 8; zz++) src[zz] = zz < splits ? cl.map_shared_rank(Ps, zz) : Ps;
    for (int q = tid; q < (jl1 - jl0) * (CB / 4); q += NT) {
      const int jl = jl0 + q / (CB / 4), b4 = (q % (CB / 4)) * 4;
      float4 sr = make_float4(0.f, 0.f, 0.f, 0.f), si = sr;
#pragma unroll
      for (int zz = 0; zz < 8; zz++) {
        if (zz < splits) {
          sr = f4add(sr, *(const float4*)(src[zz] + jl * CB + b4));
          si = f4add(si, *(const float4*)(src[zz] + CB * CB + jl * CB + b4));
        }
      }
      chain_finish(g, Rt, Ot, cs + b4, j0 + jl, m0 + b4, sr, si);
    }
    cl.sync();  // the partials stay readable until every CTA of the cluster is done
    return;
  }
  // split K: partial tile [2][CB (j)][CB (b)] to scratch, last CTA reduces
  const int tile = blockIdx.y * gridDim.x + blockIdx.x;
  float* P = part + ((long long)tile * splits + z) * 2 * CB * CB;
#pragma unroll
  for (int j = 0; j < 4; j++)
#pragma unroll
    for (int h = 0; h < TM / 4; h++) {
      *(float4*)(P + (bn + j) * CB + am + 4 * h) = quad_re(h, j);
      *(float4*)(P + CB * CB + (bn + j) * CB + am + 4 * h) = quad_im(h, j);
    }
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = atomicAdd(&cnt[tile], 1u) == (unsigned)(splits - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const float* P0 = part + (long long)tile * splits * 2 * CB * CB;
  for (int q = tid; q < CB * CB / 4; q += NT) {
    const int jl = q / (CB / 4), b4 = (q % (CB / 4)) * 4;
    float4 sr = make_float4(0.f, 0.f, 0.f, 0.f), si = sr;
#pragma unroll
    for (int zz = 0; zz < 8; zz++) {  // splits <= 8; all loads in flight at once
      if (zz < splits) {
        const float* Pz = P0 + (long long)zz * 2 * CB * CB;
        sr = f4add(sr, __ldcg((const float4*)(Pz + jl * CB + b4)));
        si = f4add(si, __ldcg((const float4*)(Pz + CB * CB + jl * CB + b4)));
      }
    }
    chain_finish(g, Rt, Ot, cs + b4, j0 + jl, m0 + b4, sr, si);
  }
  if (tid == 0) cnt[tile] = 0u;  // ready for the next launch
}

// ---------------------------------------------------------------------------
// Persistent chain: every step of the chain in one launch.  Each CTA keeps
// its output tile and K split for all steps; the split CTAs of a tile form a
// cluster and reduce through distributed shared memory as in the per-step
// kernel; between steps a grid-wide barrier (one counter, bounded wait)
// makes the step's states visible before any CTA reads them, and the next
// step's first D^T stages are fetched before the barrier.  The grid is at
// most two CTAs per SM and is launched cooperatively where possible, so all
// CTAs are resident.  A barrier that waits longer than about 2 s sets the
// timeout bit of the error word and every CTA returns.
constexpr long long kBarWaitCycles = 4000000000LL;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <bool RENORM, int TM>
__global__ void __launch_bounds__(1024 / TM, 2)
    chain32_persist_kernel(ChainDims g, int kps, const float* __restrict__ Dt0, long long dstride,
                           int steps_per_slice, int nsteps, float* __restrict__ Ra, float* __restrict__ Rb,
                           unsigned* __restrict__ bar, unsigned int* __restrict__ err) {
  constexpr int NT = 1024 / TM;
  constexpr int NQ = NT / CB;
  extern __shared__ __align__(16) float sm[];
  __shared__ float2 cs[CB];
  __shared__ float2 trp[NQ][CB];
  __shared__ int timed_out;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int tid = threadIdx.x;
  const int j0 = blockIdx.x * CB, m0 = blockIdx.y * CB, z = blockIdx.z, splits = gridDim.z;
  const int kt0 = z * kps;
  const int kt1 = min(g.Kp / CK, kt0 + kps);
  const int nkt = kt1 - kt0;
  const long long pA = (long long)g.Kp * g.Bp, pB = (long long)g.Kp * g.Np;
  const unsigned nctas = gridDim.x * gridDim.y * gridDim.z;
  const int w = tid >> 5, l = tid & 31;
  const int am = TM == 4 ? (w >> 2) * 32 + (l & 7) * 4 : (w >> 1) * 32 + (l & 3) * 8;
  const int bn = TM == 4 ? (w & 3) * 16 + (l >> 3) * 4 : (w & 1) * 32 + (l >> 2) * 4;
  const float* Dt = Dt0;
  auto loadA = [&](const float* Rt, int stage, int kt) {
    float* sA = sm + stage * STAGE_FLOATS;
    const int k0 = kt * CK;
    for (int c = tid; c < NPL * CK * (CB / 4); c += NT) {
      const int p = c / (CK * (CB / 4)), r = (c / (CB / 4)) % CK, q = c % (CB / 4);
      cp16(sA + (p * CK + r) * CB + 4 * q, Rt + p * pA + (long long)(k0 + r) * g.Bp + m0 + 4 * q);
    }
  };
  auto loadB = [&](int stage, int kt) {
    float* sB = sm + stage * STAGE_FLOATS + OPER_FLOATS;
    const int k0 = kt * CK;
    for (int c = tid; c < NPL * CK * (CB / 4); c += NT) {
      const int p = c / (CK * (CB / 4)), r = (c / (CB / 4)) % CK, q = c % (CB / 4);
      cp16(sB + (p * CK + r) * CB + 4 * q, Dt + p * pB + (long long)(k0 + r) * g.Np + j0 + 4 * q);
    }
  };
  // the first step's D^T stages
#pragma unroll
  for (int s = 0; s < CSTAGE - 1; s++)
    if (s < nkt) loadB(s, kt0 + s);
  for (int t = 0; t < nsteps; t++) {
    const float* Rt = (t & 1) ? Rb : Ra;
    float* Ot = (t & 1) ? Ra : Rb;
#pragma unroll
    for (int s = 0; s < CSTAGE - 1; s++) {
      if (s < nkt) loadA(Rt, s, kt0 + s);
      cp_commit();
    }
    if (RENORM) {
      const int b = m0 + (tid & (CB - 1)), q0 = tid / CB;
      float tr = 0.f, ti = 0.f;
      if (b < g.B) {
#pragma unroll
        for (int u = 0; u < 32 / NQ; u++) {
          const int i = q0 + NQ * u;
          if (i < g.d) {
            const long long k = (long long)i * (g.d + 1) * g.Bp + b;
            tr += __ldcg(Rt + k);
            ti += __ldcg(Rt + pA + k);
          }
        }
      }
      trp[q0][tid & (CB - 1)] = make_float2(tr, ti);
    }
    float t1[TM][4], t2[TM][4], t3[TM][4];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
      for (int j = 0; j < 4; j++) t1[i][j] = t2[i][j] = t3[i][j] = 0.f;
    for (int it = 0; it < nkt; it++) {
      cp_wait<CSTAGE - 2>();
      __syncthreads();
      {
        const int nx = it + CSTAGE - 1;
        if (nx < nkt) {
          loadA(Rt, nx % CSTAGE, kt0 + nx);
          loadB(nx % CSTAGE, kt0 + nx);
        }
        cp_commit();
      }
      const float* sA = sm + (it % CSTAGE) * STAGE_FLOATS;
      const float* sB = sA + OPER_FLOATS;
      constexpr int QA = TM / 4;
      float4 fa[2][NPL][QA], fb[2][NPL];
#pragma unroll
      for (int p = 0; p < NPL; p++) {
#pragma unroll
        for (int h = 0; h < QA; h++) fa[0][p][h] = *(const float4*)(sA + (p * CK) * CB + am + 4 * h);
        fb[0][p] = *(const float4*)(sB + (p * CK) * CB + bn);
      }
#pragma unroll
      for (int k = 0; k < CK; k++) {
        const int cur = k & 1;
        if (k + 1 < CK) {
#pragma unroll
          for (int p = 0; p < NPL; p++) {
#pragma unroll
            for (int h = 0; h < QA; h++)
              fa[cur ^ 1][p][h] = *(const float4*)(sA + (p * CK + k + 1) * CB + am + 4 * h);
            fb[cur ^ 1][p] = *(const float4*)(sB + (p * CK + k + 1) * CB + bn);
          }
        }
        float ar[TM], ai[TM], as[TM];
#pragma unroll
        for (int h = 0; h < QA; h++) {
          ar[4 * h] = fa[cur][0][h].x; ar[4 * h + 1] = fa[cur][0][h].y;
          ar[4 * h + 2] = fa[cur][0][h].z; ar[4 * h + 3] = fa[cur][0][h].w;
          ai[4 * h] = fa[cur][1][h].x; ai[4 * h + 1] = fa[cur][1][h].y;
          ai[4 * h + 2] = fa[cur][1][h].z; ai[4 * h + 3] = fa[cur][1][h].w;
        }
#pragma unroll
        for (int i = 0; i < TM; i++) as[i] = ar[i] + ai[i];
        const float br[4] = {fb[cur][0].x, fb[cur][0].y, fb[cur][0].z, fb[cur][0].w};
        const float bi[4] = {fb[cur][1].x, fb[cur][1].y, fb[cur][1].z, fb[cur][1].w};
        const float bs[4] = {br[0] + bi[0], br[1] + bi[1], br[2] + bi[2], br[3] + bi[3]};
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
          for (int j = 0; j < 4; j++) {
            t1[i][j] = fmaf(ar[i], br[j], t1[i][j]);
            t2[i][j] = fmaf(ai[i], bi[j], t2[i][j]);
            t3[i][j] = fmaf(as[i], bs[j], t3[i][j]);
          }
      }
    }
    cp_wait<0>();
    __syncthreads();
    if (tid < CB) {
      float2 c = make_float2(0.f, 0.f);
      if (m0 + tid < g.B) {
        if (RENORM) {
          float tr = 0.f, ti = 0.f;
#pragma unroll
          for (int q = 0; q < NQ; q++) {
            tr += trp[q][tid].x;
            ti += trp[q][tid].y;
          }
          const float m2 = tr * tr + ti * ti;
          c = make_float2(tr / m2, -ti / m2);
        } else {
          c = make_float2(1.f, 0.f);
        }
      }
      cs[tid] = c;
    }
    // partial tile in the (idle) ring; CTA r of the cluster finishes its
    // share of the tile's rows over all partials, in split order
    float* Ps = sm;
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int h = 0; h < TM / 4; h++) {
        float4 qr, qi;
        qr.x = t1[4 * h][j] - t2[4 * h][j];
        qr.y = t1[4 * h + 1][j] - t2[4 * h + 1][j];
        qr.z = t1[4 * h + 2][j] - t2[4 * h + 2][j];
        qr.w = t1[4 * h + 3][j] - t2[4 * h + 3][j];
        qi.x = t3[4 * h][j] - t1[4 * h][j] - t2[4 * h][j];
        qi.y = t3[4 * h + 1][j] - t1[4 * h + 1][j] - t2[4 * h + 1][j];
        qi.z = t3[4 * h + 2][j] - t1[4 * h + 2][j] - t2[4 * h + 2][j];
        qi.w = t3[4 * h + 3][j] - t1[4 * h + 3][j] - t2[4 * h + 3][j];
        *(float4*)(Ps + (bn + j) * CB + am + 4 * h) = qr;
        *(float4*)(Ps + CB * CB + (bn + j) * CB + am + 4 * h) = qi;
      }
    cl.sync();
    {
      const int rank = (int)cl.block_rank();
      const int rows = (CB + splits - 1) / splits;
      const int jl0 = rank * rows, jl1 = min(CB, jl0 + rows);
      const float* src[8];
#pragma unroll
      for (int zz = 0; zz < 8; zz++) src[zz] = zz < splits ? cl.map_shared_rank(Ps, zz) : Ps;
      for (int q = tid; q < (jl1 - jl0) * (CB / 4); q += NT) {
        const int jl = jl0 + q / (CB / 4), b4 = (q % (CB / 4)) * 4;
        float4 sr = make_float4(0.f, 0.f, 0.f, 0.f), si = sr;
#pragma unroll
        for (int zz = 0; zz < 8; zz++) {
          if (zz < splits) {
            sr = f4add(sr, *(const float4*)(src[zz] + jl * CB + b4));
            si = f4add(si, *(const float4*)(src[zz] + CB * CB + jl * CB + b4));
          }
        }
        chain_finish(g, Rt, Ot, cs + b4, j0 + jl, m0 + b4, sr, si);
      }
    }
    cl.sync();  // the partials stay readable until every CTA of the cluster is done
    if (t + 1 == nsteps) break;
    // the next step's D^T stages (written before the chain), then the grid
    // barrier: every tile of O_t written before anyone reads it.  Each CTA
    // arrives; rank 0 of the cluster waits for all and hands its verdict to
    // the cluster, so a timeout ends whole clusters (no CTA is left waiting
    // at a cluster barrier for one that returned).
    Dt = Dt0 + (long long)((t + 1) / steps_per_slice) * dstride;
#pragma unroll
    for (int s = 0; s < CSTAGE - 1; s++)
      if (s < nkt) loadB(s, kt0 + s);
    if (tid == 0) {
      __threadfence();
      atomicAdd(bar, 1u);
      if (cl.block_rank() == 0) {
        const unsigned target = (unsigned)(t + 1) * nctas;
        int to = 0;
        if (ld_acquire_u32(bar) < target) {
          const long long c0 = clock64();
          while (ld_acquire_u32(bar) < target) {
            if (clock64() - c0 > kBarWaitCycles) {
              to = 1;
              atomicOr(err, ERR_TIMEOUT);
              break;
            }
          }
        }
        __threadfence();
        for (int r = 0; r < splits; r++) *cl.map_shared_rank(&timed_out, r) = to;
      }
    }
    cl.sync();
    if (timed_out) {
      cp_wait<0>();
      return;
    }
  }
}

// D^T planes of S propagators: Dt[s][p][k][j] = (P_s - I)[j][k], zero padding.
__global__ void chain32_dplanes_kernel(int n, int Kp, int Np, const z64* __restrict__ P, float* __restrict__ Dt) {
  __shared__ float tr[32][33], ti[32][33];
  const long long nn = (long long)n * n;
  const z64* Ps = P + blockIdx.z * nn;
  float* D = Dt + (long long)blockIdx.z * NPL * Kp * Np;
  const long long pl = (long long)Kp * Np;
  const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32, tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, k = k0 + tx;
    double vr = 0.0, vi = 0.0;
    if (j < n && k < n) {
      const z64 v = Ps[(long long)j * n + k];
      vr = v.x - (j == k ? 1.0 : 0.0);
      vi = v.y;
    }
    tr[r][tx] = (float)vr;
    ti[r][tx] = (float)vi;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, j = j0 + tx;
    if (k >= Kp || j >= Np) continue;
    const float a = tr[tx][r], b = ti[tx][r];
    const long long idx = (long long)k * Np + j;
    D[idx] = a;
    D[pl + idx] = b;
  }
}

// states (B x n, complex128) -> Rt planes, every element of [2][Kp][Bp] written.
__global__ void chain32_states_in_kernel(int n, int B, int Kp, int Bp, const z64* __restrict__ X,
                                         float* __restrict__ Rt) {
  __shared__ float tr[32][33], ti[32][33];
  const long long pl = (long long)Kp * Bp;
  const int b0 = blockIdx.x * 32, k0 = blockIdx.y * 32, tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int b = b0 + r, k = k0 + tx;
    z64 v = make_double2(0.0, 0.0);
    if (b < B && k < n) v = X[(long long)b * n + k];
    tr[r][tx] = (float)v.x;
    ti[r][tx] = (float)v.y;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, b = b0 + tx;
    if (k >= Kp || b >= Bp) continue;
    const float a = tr[tx][r], c = ti[tx][r];
    const long long idx = (long long)k * Bp + b;
    Rt[idx] = a;
    Rt[pl + idx] = c;
  }
}

// Rt planes -> states (B x n, complex128), divided by the trace if asked.
__global__ void chain32_states_out_kernel(int n, int d, int B, int Kp, int Bp, int renorm,
                                          const float* __restrict__ Rt, z64* __restrict__ X) {
  __shared__ float tr[32][33], ti[32][33];
  __shared__ float2 cs[32];
  const long long pl = (long long)Kp * Bp;
  const int b0 = blockIdx.x * 32, k0 = blockIdx.y * 32, tx = threadIdx.x;
  if (threadIdx.y == 0) {
    float2 c = make_float2(1.f, 0.f);
    const int b = b0 + tx;
    if (renorm && b < B) {
      float sr = 0.f, si = 0.f;
      for (int i = 0; i < d; i++) {
        const long long k = (long long)i * (d + 1) * Bp + b;
        sr += Rt[k];
        si += Rt[pl + k];
      }
      const float m2 = sr * sr + si * si;
      c = make_float2(sr / m2, -si / m2);
    }
    cs[tx] = c;
  }
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, b = b0 + tx;
    float a = 0.f, c = 0.f;
    if (k < n && b < B) {
      a = Rt[(long long)k * Bp + b];
      c = Rt[pl + (long long)k * Bp + b];
    }
    tr[r][tx] = a;
    ti[r][tx] = c;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int b = b0 + r, k = k0 + tx;
    if (b >= B || k >= n) continue;
    const float a = tr[tx][r], c = ti[tx][r];
    const float2 s = cs[r];
    X[(long long)b * n + k] = make_double2((double)(a * s.x - c * s.y), (double)(a * s.y + c * s.x));
  }
}

int rup(int x, int m) { return (x + m - 1) / m * m; }

// Whether `tiles` clusters of `splits` CTAs of this kernel can be resident at
// once (queried once per kernel, device and cluster size).
template <typename Kern>
bool cluster_fits(Kern kern, int splits, int tiles) {
  constexpr int NT = 1024 / kChainTM;
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple((const void*)kern, dev, splits);
  auto it = cache.find(key);
  if (it == cache.end()) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, 1, splits);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = STEP_SMEM;
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeClusterDimension;
    a.val.clusterDim.x = 1;
    a.val.clusterDim.y = 1;
    a.val.clusterDim.z = splits;
    cfg.attrs = &a;
    cfg.numAttrs = 1;
    int num = 0;
    if (set_smem_once((const void*)kern, STEP_SMEM) != cudaSuccess ||
        cudaOccupancyMaxActiveClusters(&num, (const void*)kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      num = 0;
    }
    it = cache.emplace(key, num).first;
  }
  return it->second >= tiles;
}

int chain_isqrt(int n) {
  int d = 1;
  while ((d + 1) * (d + 1) <= n) d++;
  return d;
}

}  // namespace

size_t chain32_dplane_floats(int n) { return (size_t)NPL * rup(n, CK) * rup(n, CB); }
size_t chain32_state_floats(int n, int B) { return (size_t)NPL * rup(n, CK) * rup(B, CB); }
size_t chain32_part_floats(int sm_count) { return (size_t)2 * sm_count * 2 * CB * CB; }

cudaError_t launch_chain32_dplanes(int n, int S, const z64* P, float* Dt, cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  const int Kp = rup(n, CK), Np = rup(n, CB);
  dim3 grid(Np / 32, (Kp + 31) / 32, S), block(32, 8);
  count_launch();
  chain32_dplanes_kernel<<<grid, block, 0, st>>>(n, Kp, Np, P, Dt);
  return cudaGetLastError();
}

cudaError_t launch_chain32_states_in(int n, int B, const z64* X, float* Rt, cudaStream_t st) {
  const int Kp = rup(n, CK), Bp = rup(B, CB);
  dim3 grid(Bp / 32, (Kp + 31) / 32), block(32, 8);
  count_launch();
  chain32_states_in_kernel<<<grid, block, 0, st>>>(n, B, Kp, Bp, X, Rt);
  return cudaGetLastError();
}

cudaError_t launch_chain32_states_out(int n, int B, int renorm, const float* Rt, z64* X, cudaStream_t st) {
  const int Kp = rup(n, CK), Bp = rup(B, CB);
  dim3 grid(Bp / 32, (n + 31) / 32), block(32, 8);
  count_launch();
  chain32_states_out_kernel<<<grid, block, 0, st>>>(n, chain_isqrt(n), B, Kp, Bp, renorm, Rt, X);
  return cudaGetLastError();
}

bool launch_chain32_persist(int n, int B, int renorm, const float* Dt, long long dstride, int steps_per_slice,
                            int nsteps, float* Ra, float* Rb, unsigned* bar, unsigned int* err, int sm_count,
                            cudaStream_t st, cudaError_t* status) {
  *status = cudaSuccess;
  ChainDims g;
  g.n = n;
  g.d = chain_isqrt(n);
  g.B = B;
  g.Kp = rup(n, CK);
  g.Np = rup(n, CB);
  g.Bp = rup(B, CB);
  const int tilesN = g.Np / CB, tilesM = g.Bp / CB, tiles = tilesN * tilesM;
  const int ktiles = g.Kp / CK;
  if (nsteps < 2 || tiles >= sm_count) return false;
  void (*kern)(ChainDims, int, const float*, long long, int, int, float*, float*, unsigned*, unsigned int*) =
      renorm ? chain32_persist_kernel<true, kChainTM> : chain32_persist_kernel<false, kChainTM>;
  // the per-step launches' K split (at most two CTAs per SM, four K blocks
  // per split), if its clusters all fit at once; a narrower split gives
  // each CTA more of the K loop per step and was measured slower than the
  // per-step launches with the wide split (256 states: 7.2 against 6.5 ms)
  const int want = std::max(1, std::min({2 * sm_count / tiles, ktiles / 4, 8}));
  const int kps = (ktiles + want - 1) / want;
  const int splits = (ktiles + kps - 1) / kps;
  if (splits < 2 || tiles * splits > 2 * sm_count || !cluster_fits(kern, splits, tiles)) return false;
  // whether a cooperative cluster launch of this kernel was accepted on this
  // device: tried outside stream capture only (a refused launch would end a
  // capture), remembered for captures
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int>, int> accepted;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple((const void*)kern, dev, splits);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = accepted.find(key);
    if (it != accepted.end() && it->second == 0) return false;
    if (it == accepted.end() && cap != cudaStreamCaptureStatusNone) return false;
  }
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) {
    *status = e;
    return true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tilesN, tilesM, splits);
  cfg.blockDim = dim3(1024 / kChainTM);
  cfg.dynamicSmemBytes = STEP_SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = splits;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  e = cudaLaunchKernelEx(&cfg, kern, g, kps, Dt, dstride, steps_per_slice, nsteps, Ra, Rb, bar, err);
  std::lock_guard<std::mutex> lk(mu);
  if (e != cudaSuccess) {  // refused (not in a capture, see above): per-step launches from now on
    cudaGetLastError();
    accepted[key] = 0;
    return false;
  }
  accepted[key] = 1;
  count_launch();
  return true;
}

cudaError_t launch_chain32_step(int n, int B, int renorm, const float* Dt, const float* Rt, float* Ot, float* part,
                                unsigned* cnt, int sm_count, bool pdl, cudaStream_t st) {
  ChainDims g;
  g.n = n;
  g.d = chain_isqrt(n);
  g.B = B;
  g.Kp = rup(n, CK);
  g.Np = rup(n, CB);
  g.Bp = rup(B, CB);
  const int tilesN = g.Np / CB, tilesM = g.Bp / CB, tiles = tilesN * tilesM;
  const int ktiles = g.Kp / CK;
  // two CTAs fit on an SM: split K until the grid fills them (at least four
  // K blocks per split)
  int splits = 1;
  if (tiles < 2 * sm_count) splits = std::max(1, std::min({2 * sm_count / tiles, ktiles / 4, 8}));
  const int kps = (ktiles + splits - 1) / splits;
  splits = (ktiles + kps - 1) / kps;
  if (splits > 1 && (tiles * splits > 2 * sm_count || tiles > sm_count))
    return cudaErrorInvalidValue;  // scratch is sized for 2 x sm_count partial tiles, sm_count tickets
  void (*kern)(ChainDims, int, const float*, const float*, float*, float*, unsigned*, int) =
      renorm ? chain32_step_kernel<true, kChainTM> : chain32_step_kernel<false, kChainTM>;
  cudaError_t e = set_smem_once((const void*)kern, STEP_SMEM);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tilesN, tilesM, splits);
  cfg.blockDim = dim3(1024 / kChainTM);
  cfg.dynamicSmemBytes = STEP_SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  // the split CTAs of a tile as one cluster, if that many clusters fit at once
  const bool cluster = splits > 1 && cluster_fits(kern, splits, tiles);
  if (cluster) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = 1;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = splits;
    na++;
  }
  if (pdl) {  // only after another step (the D^T planes must be complete)
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    na++;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, g, kps, Dt, Rt, Ot, part, cnt, cluster ? 1 : 0);
}

}  // namespace lb
