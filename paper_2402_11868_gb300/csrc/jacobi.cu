// Batched complex Hermitian FP64 Jacobi eigensolver: the double-precision diagonalisation stage that
// precedes precision recovery (Section 2, ZKCM_CUS paragraph: a double-precision eigensolve whose
// result Rayleigh quotient iteration then refines).  The paper calls a cuSOLVER routine here; this is a
// hand-written two-sided Jacobi method instead.
//
// Parallel ordering: a sweep has m-1 rounds (m = n rounded up to even); in a round the m/2 disjoint
// pairs of the circle method rotate at once.  For pair k = (p, q) with b = a_pq = |b| e^{i phi}:
//   tau = (a_qq - a_pp) / (2|b|), t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c,
//   J_k = [[c, z2], [-z1, c]] with z1 = s e^{-i phi}, z2 = s e^{i phi}.
// The whole round is A <- J^H A J with J = prod_k J_k.  It is applied as 2x2-block updates
//   A[{p,q},{p',q'}] <- J_k^H A[{p,q},{p',q'}] J_k'
// on the upper block triangle k <= k' (the lower one is its conjugate transpose), so one barrier per
// round suffices and Hermitian symmetry halves the arithmetic; diagonal blocks use the closed form
// (a_pp - t|b|, a_qq + t|b|, 0).  V <- V J accumulates the eigenvectors.
// Rotations with |a_pq| <= tol = sqrt(n) 2^-53 ||A||_F are skipped; a sweep without rotation ends the
// iteration.  Output: eigenvalues descending, eigenvectors with their first largest-modulus component
// real and positive.
#include "common.cuh"
#include "mw.cuh"
#include "prof.cuh"
#include "internal.cuh"
#include <cooperative_groups.h>
namespace cg = cooperative_groups;

namespace zkq {

// Rotations act on scaled matrices (fast rotations): the true A_ij = s_i s_j A~_ij and V_ij = V~_ij s_j
// with a positive scale s per index.  Rotating the pair (p, q) multiplies s_p and s_q by c, so the stored
// entries take the rotation divided by c, I + w: col p -= w1 col q, col q += w2 col p (and the conjugate
// transpose from the left) with w1 = t e^{-i phi} s_q / s_p, w2 = t e^{i phi} s_p / s_q, |t| <= 1.  That is
// 4 FMA per complex entry instead of 6.  The scales are folded back into A~ and V~ after every 256 rounds
// and at the end of every sweep.
// Stored per pair: c, the new stored diagonal entries dpn, dqn (true values over the new squared scales).
struct RotParams { double c, dpn, dqn; c64 w1, w2; int rot; int p, q; };

// x - w y, x + w y, x - conj(w) y, x + conj(w) y with four FMA each
__device__ __forceinline__ c64 c_sub_mul(c64 x, c64 w, c64 y) {
  return {fma(-w.re, y.re, fma(w.im, y.im, x.re)), fma(-w.re, y.im, fma(-w.im, y.re, x.im))};
}
__device__ __forceinline__ c64 c_add_mul(c64 x, c64 w, c64 y) {
  return {fma(w.re, y.re, fma(-w.im, y.im, x.re)), fma(w.re, y.im, fma(w.im, y.re, x.im))};
}
__device__ __forceinline__ c64 c_sub_cmul(c64 x, c64 w, c64 y) {
  return {fma(-w.re, y.re, fma(-w.im, y.im, x.re)), fma(-w.re, y.im, fma(w.im, y.re, x.im))};
}
__device__ __forceinline__ c64 c_add_cmul(c64 x, c64 w, c64 y) {
  return {fma(w.re, y.re, fma(w.im, y.im, x.re)), fma(w.re, y.im, fma(-w.im, y.re, x.im))};
}


// Storage policy: matrix element (i, j) of a column-major matrix with leading dimension ld.
// SMEM: plain loads/stores.  GLOBAL: L2-only loads (other CTAs of the cluster write the same matrix).
template <bool SMEM> struct Mat {
  c64* base; int ld;
  __device__ __forceinline__ c64 get(int i, int j) const {
    if (SMEM) return base[i + (size_t)j * ld];
    const double2 v = __ldcg(reinterpret_cast<const double2*>(base + i + (size_t)j * ld));
    return {v.x, v.y};
  }
  __device__ __forceinline__ void set(int i, int j, c64 v) const {
    if (SMEM) base[i + (size_t)j * ld] = v;
    else __stcg(reinterpret_cast<double2*>(base + i + (size_t)j * ld), make_double2(v.re, v.im));
  }
};

// One problem, processed by `nparts` cooperating CTAs: a thread-block cluster (SYNC 1), the whole grid of
// a cooperative launch (SYNC 2), or a single CTA (SYNC 0, nparts = 1).
__device__ __forceinline__ void cluster_barrier() { __threadfence(); cg::this_cluster().sync(); }

// Test hook of the grid barrier (zkq_test_grid_barrier_hook): `extra` arrivals that never come (the barrier
// then waits on a generation flag that nothing advances) and the log2 of the poll limit.  Defaults: none, 2^22.
struct WaitHook { int extra; int log2_limit; };
__device__ WaitHook g_wait_hook = {0, 22};

// Grid barrier of a cooperative launch (all blocks co-resident): arrival counter + generation number.  The
// wait is bounded; on expiry the barrier raises gb->abort, after which no barrier waits any more, so every
// block runs its remaining (bounded) loops to the end and the problem reports failure.
__device__ __forceinline__ void grid_barrier(GridBar* gb, unsigned nblocks) {
  __syncthreads();
  if (threadIdx.x == 0 && !*(volatile int*)&gb->abort) {
    const WaitHook hook = g_wait_hook;
    __threadfence();
    const unsigned g = *(volatile unsigned*)&gb->gen;
    if (atomicAdd(&gb->count, 1u) == nblocks - 1 + (unsigned)hook.extra) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      for (int it = 0; *(volatile unsigned*)&gb->gen == g; ++it) {
        if (it > (1 << hook.log2_limit)) { atomicExch(&gb->abort, 1); break; }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

template <bool SMEM, int SYNC, int WA>
__device__ void jacobi_problem(int n, const double* __restrict__ A_in, Mat<SMEM> A, Mat<SMEM> V,
                               RotParams* rp, double* sig, double* red, int max_sweeps, unsigned long long* flops,
                               double* __restrict__ W_out, double* __restrict__ V_out, int32_t* info,
                               int part, int nparts, GridBar* gb = nullptr) {
  auto sync = [&] {
    if constexpr (SYNC == 1) cluster_barrier();
    else if constexpr (SYNC == 2) grid_barrier(gb, (unsigned)nparts);
    else __syncthreads();
  };
  const int tid = threadIdx.x, nth = blockDim.x;
  const int gtid = part * nth + tid, gnth = nparts * nth;
  const int m = n + (n & 1);               // even number of players; index n is a dummy when n is odd
  const int P = m / 2;
  // load A (leading word of each real part; the expansions are normalised so it is the nearest double)
  double fro_part = 0.0;
  for (int e = gtid; e < n * n; e += gnth) {
    int i = e % n, j = e / n;
    const double* q = A_in + (size_t)e * 2 * WA;
    c64 v = {q[0], q[WA]};
    if (i == j) v.im = 0.0;
    A.set(i, j, v);
    V.set(i, j, c64{i == j ? 1.0 : 0.0, 0.0});
    fro_part += v.re * v.re + v.im * v.im;
  }
  for (int i = tid; i < n; i += nth) sig[i] = 1.0;   // every CTA keeps its own copy of the scales
  // ||A||_F: block reduction; with several CTAs each keeps its own partial, combined via red[] in global
  __shared__ double s_red[32];
  __shared__ double s_tol;
  __shared__ int s_rot;
  for (int o = 16; o > 0; o >>= 1) fro_part += __shfl_down_sync(0xffffffffu, fro_part, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = fro_part;
  __syncthreads();
  if (tid == 0) {
    double s = 0; for (int w = 0; w < (nth + 31) / 32; ++w) s += s_red[w];
    if (nparts > 1) red[part] = s; else s_tol = s;
  }
  sync();
  if (tid == 0) {
    double s = s_tol;
    if (nparts > 1) { s = 0; for (int k = 0; k < nparts; ++k) s += __ldcg(red + k); }
    s_tol = sqrt((double)n) * 0x1p-53 * sqrt(s);
  }
  __syncthreads();
  const double tol = s_tol;
  int sweep = 0, converged = 0;
  for (sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    int my_rot = 0;
    for (int r = 0; r < m - 1; ++r) {
      // phase 1: rotation parameters.  A cluster's CTAs split the pairs: each computes its share into a
      // staging area of its shared memory, and after the cluster barrier every CTA copies all pairs from
      // their owners (distributed shared memory).  The staging area is rewritten only after the next
      // cluster barrier, by which time every copy of it is done.  A single CTA, or the blocks of a
      // cooperative grid (no distributed shared memory), compute every pair themselves.
      const int per = SYNC == 1 ? (P + nparts - 1) / nparts : P;
      const int k0 = SYNC == 1 ? part * per : 0, k1 = min(P, k0 + per);
      RotParams* stage = SYNC == 1 ? rp + P : rp;
      for (int k = k0 + tid; k < k1; k += nth) {
        int p, q; rr_pair(m, r, k, p, q);
        RotParams pr; pr.p = p; pr.q = q; pr.rot = 0; pr.c = 1.0; pr.dpn = 0.0; pr.dqn = 0.0; pr.w1 = {0, 0}; pr.w2 = {0, 0};
        if (q < n) {
          const double sp = sig[p], sq = sig[q];
          const c64 bs = A.get(p, q);
          const c64 b = {bs.re * (sp * sq), bs.im * (sp * sq)};      // true entries
          double ab = hypot(b.re, b.im);
          if (ab > tol) {
            double app = A.get(p, p).re * (sp * sp), aqq = A.get(q, q).re * (sq * sq);
            double tau = (aqq - app) / (2.0 * ab);
            double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            double c = 1.0 / sqrt(1.0 + t * t);
            double er = b.re / ab, ei = b.im / ab;
            const double tb = t * ab, rq = sq / sp;
            pr.c = c; pr.rot = 1;
            pr.w1 = {t * er * rq, -t * ei * rq};
            pr.w2 = {t * er / rq, t * ei / rq};
            pr.dpn = (app - tb) / ((c * sp) * (c * sp));             // (a_pp - t|b|) / s_p'^2
            pr.dqn = (aqq + tb) / ((c * sq) * (c * sq));
          }
        }
        stage[k - k0] = pr;
        if (SYNC != 1) my_rot += pr.rot;
      }
      sync();
      if constexpr (SYNC == 1) {
        cg::cluster_group cl = cg::this_cluster();
        for (int k = tid; k < P; k += nth) {
          const int owner = k / per;
          const RotParams* src = cl.map_shared_rank(rp + P, owner);
          const RotParams pr = src[k - owner * per];
          rp[k] = pr;
          my_rot += pr.rot;                        // every CTA counts all pairs: the same total everywhere
          if (pr.rot) { sig[pr.p] *= pr.c; sig[pr.q] *= pr.c; }   // pairs are disjoint: no conflicts
        }
        __syncthreads();
      } else {
        for (int k = tid; k < P; k += nth) {
          const RotParams& pr = rp[k];
          if (pr.rot) { sig[pr.p] *= pr.c; sig[pr.q] *= pr.c; }
        }
      }
      // phase 2: 2x2 block updates on the upper block triangle + V <- V J
      const int nblk = P * (P + 1) / 2;
      for (int it = gtid; it < nblk + n * P; it += gnth) {
        if (it < nblk) {
          // decode (k, k2) with k <= k2 from the linear index
          int k = (int)((sqrtf(8.0f * (float)it + 1.0f) - 1.0f) * 0.5f);
          while ((k + 1) * (k + 2) / 2 <= it) ++k;
          while (k * (k + 1) / 2 > it) --k;
          int k2 = it - k * (k + 1) / 2;           // k2 <= k
          const RotParams a = rp[k2], b = rp[k];   // rows from pair k2, columns from pair k
          if (k2 == k) {
            if (a.rot) {
              A.set(a.p, a.p, c64{a.dpn, 0.0});
              A.set(a.q, a.q, c64{a.dqn, 0.0});
              A.set(a.p, a.q, c64{0.0, 0.0});
              A.set(a.q, a.p, c64{0.0, 0.0});
            }
            continue;
          }
          if (!a.rot && !b.rot) continue;
          const int r0 = a.p, r1 = a.q, c0 = b.p, c1 = b.q;
          const bool hr1 = r1 < n, hc1 = c1 < n;
          c64 x00 = A.get(r0, c0);
          c64 x01 = hc1 ? A.get(r0, c1) : c64{0, 0};
          c64 x10 = hr1 ? A.get(r1, c0) : c64{0, 0};
          c64 x11 = (hr1 && hc1) ? A.get(r1, c1) : c64{0, 0};
          // T = X (I + W_b): col0 = X[:,0] - w1 X[:,1], col1 = X[:,1] + w2 X[:,0]
          c64 t00, t01, t10, t11;
          if (b.rot) {
            t00 = c_sub_mul(x00, b.w1, x01); t01 = c_add_mul(x01, b.w2, x00);
            t10 = c_sub_mul(x10, b.w1, x11); t11 = c_add_mul(x11, b.w2, x10);
          } else { t00 = x00; t01 = x01; t10 = x10; t11 = x11; }
          // Y = (I + W_a)^H T: row0 = T[0,:] - conj(w1) T[1,:], row1 = T[1,:] + conj(w2) T[0,:]
          c64 y00, y01, y10, y11;
          if (a.rot) {
            y00 = c_sub_cmul(t00, a.w1, t10); y10 = c_add_cmul(t10, a.w2, t00);
            y01 = c_sub_cmul(t01, a.w1, t11); y11 = c_add_cmul(t11, a.w2, t01);
          } else { y00 = t00; y01 = t01; y10 = t10; y11 = t11; }
          A.set(r0, c0, y00); A.set(c0, r0, cconj(y00));
          if (hc1) { A.set(r0, c1, y01); A.set(c1, r0, cconj(y01)); }
          if (hr1) { A.set(r1, c0, y10); A.set(c0, r1, cconj(y10)); }
          if (hr1 && hc1) { A.set(r1, c1, y11); A.set(c1, r1, cconj(y11)); }
        } else {
          int e = it - nblk;
          int i = e % n, k = e / n;
          const RotParams b = rp[k];
          if (!b.rot) continue;
          c64 x = V.get(i, b.p), y = V.get(i, b.q);
          V.set(i, b.p, c_sub_mul(x, b.w1, y));
          V.set(i, b.q, c_add_mul(y, b.w2, x));
        }
      }
      sync();
      // fold the scales into the stored matrices after every 256 rounds and at the end of the sweep (each
      // CTA its share of the entries, with its own copy of the scales, identical in every CTA): c >= 2^-1/2,
      // so the scales stay above 2^-128 and the stored entries below 2^256 times their true size
      if ((r & 255) == 255 || r == m - 2) {
        for (int e = gtid; e < n * n; e += gnth) {
          const int i = e % n, j = e / n;
          const double sa = sig[i] * sig[j], sv = sig[j];
          const c64 a = A.get(i, j), v = V.get(i, j);
          A.set(i, j, c64{a.re * sa, a.im * sa});
          V.set(i, j, c64{v.re * sv, v.im * sv});
        }
        __syncthreads();
        for (int i = tid; i < n; i += nth) sig[i] = 1.0;
        sync();
      }
    }
    if (my_rot) atomicAdd(&s_rot, my_rot);
    __syncthreads();
    // FP64 flops of this sweep: per applied rotation 16 n FMA (8 n on A: a round's n/2 rotations update
    // n^2/8 2x2 blocks at 32 FMA each; 8 n on V) = 32 n flops; counted once per problem
    if (part == 0 && tid == 0 && flops && s_rot) atomicAdd(flops, (unsigned long long)s_rot * 32ULL * (unsigned long long)n);
    if constexpr (SYNC != 0) {
      // every CTA computed the same parameters, but take part 0's count so the barrier counts of the
      // cooperating CTAs cannot diverge
      if (tid == 0) red[nparts + part] = (double)s_rot;
      sync();
      converged = (__ldcg(red + nparts) == 0.0);
      sync();
    } else {
      converged = (s_rot == 0);
    }
    __syncthreads();
  }
  // eigenvalues: rank sort (descending, ties by index), then eigenvector phase normalisation
  for (int i = gtid; i < n; i += gnth) {
    double li = A.get(i, i).re;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double lj = A.get(j, j).re;
      rank += (lj > li) || (lj == li && j < i);
    }
    W_out[rank] = li;
    // phase: first index with the largest modulus
    int best = 0; double bm = -1.0;
    for (int r = 0; r < n; ++r) { c64 v = V.get(r, i); double m2 = v.re * v.re + v.im * v.im; if (m2 > bm) { bm = m2; best = r; } }
    c64 vb = V.get(best, i);
    double inv = 1.0 / sqrt(bm);
    c64 ph = {vb.re * inv, -vb.im * inv};    // conj(v_best)/|v_best|
    for (int r = 0; r < n; ++r) {
      c64 v = cmul(V.get(r, i), ph);
      if (r == best) v.im = 0.0;
      V_out[((size_t)r + (size_t)rank * n) * 2 + 0] = v.re;
      V_out[((size_t)r + (size_t)rank * n) * 2 + 1] = v.im;
    }
  }
  if (part == 0 && tid == 0) {
    bool failed = false;
    if constexpr (SYNC == 2) failed = *(volatile int*)&gb->abort != 0;
    *info = failed ? -1 : (converged ? 0 : sweep);
  }
}

// shared-memory bytes of the scales of an order-n problem, 16-byte aligned (the pair parameters follow)
__host__ __device__ __forceinline__ size_t jacobi_scale_bytes(int n) { return ((size_t)n * sizeof(double) + 15) & ~(size_t)15; }

// small problems: matrix and eigenvectors in shared memory, one CTA per problem
template <int WA>
__global__ void __launch_bounds__(256) jacobi_smem_kernel(JacobiBatch jb, int first, int count) {
  extern __shared__ __align__(16) unsigned char smem[];
  if ((int)blockIdx.x >= count) return;
  const int b = jb.order[first + blockIdx.x];
  const int n = jb.n[b];
  const int ld = n + 1;                       // padding avoids bank conflicts on row access
  c64* sA = reinterpret_cast<c64*>(smem);
  c64* sV = sA + (size_t)ld * n;
  RotParams* rp = reinterpret_cast<RotParams*>(sV + (size_t)ld * n);
  double* sig = reinterpret_cast<double*>(rp + (n / 2 + 1));
  Mat<true> A{sA, ld}, V{sV, ld};
  jacobi_problem<true, 0, WA>(n, jb.A + jb.a_off[b] * 2 * WA, A, V, rp, sig, nullptr, jb.max_sweeps, jb.flops,
                                  jb.W + jb.w_off[b], jb.V + jb.a_off[b] * 2, jb.info + b, 0, 1);
}

// large problems: matrix and eigenvectors in global workspace, one cluster of CTAs per problem
template <int WA>
__global__ void __launch_bounds__(256, 4) jacobi_global_kernel(JacobiBatch jb, int first) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int part = (int)cl.block_rank(), nparts = (int)cl.num_blocks();
  const int b = jb.order[first + blockIdx.x / nparts];
  const int n = jb.n[b];
  double* wsA = jb.ws + jb.ws_off[b];
  double* wsV = wsA + (size_t)n * n * 2;
  double* sig = reinterpret_cast<double*>(smem);                 // scales, then the pair parameters
  RotParams* rp = reinterpret_cast<RotParams*>(smem + jacobi_scale_bytes(n));
  Mat<false> A{reinterpret_cast<c64*>(wsA), n}, V{reinterpret_cast<c64*>(wsV), n};
  double* red = jb.red + (size_t)64 * (blockIdx.x / nparts);   // 2 * cluster (<= 32) entries used
  if (nparts > 1)
    jacobi_problem<false, 1, WA>(n, jb.A + jb.a_off[b] * 2 * WA, A, V, rp, sig, red, jb.max_sweeps, jb.flops,
                                    jb.W + jb.w_off[b], jb.V + jb.a_off[b] * 2, jb.info + b, part, nparts);
  else
    jacobi_problem<false, 0, WA>(n, jb.A + jb.a_off[b] * 2 * WA, A, V, rp, sig, red, jb.max_sweeps, jb.flops,
                                     jb.W + jb.w_off[b], jb.V + jb.a_off[b] * 2, jb.info + b, 0, 1);
}

// few large problems: a cooperative launch whose blocks form one group per problem, blocks
// grp_start[q] .. grp_start[q+1]-1 for problem q, each group with its own barrier and reduction slots
template <int WA>
__global__ void __launch_bounds__(256, 4) jacobi_grid_kernel(JacobiBatch jb, int first, int count, GridBar* gb,
                                                          const int32_t* __restrict__ grp_start, int red_stride) {
  extern __shared__ __align__(16) unsigned char smem[];
  int q = 0;
  while (q + 1 < count && (int)blockIdx.x >= grp_start[q + 1]) ++q;
  const int part = (int)blockIdx.x - grp_start[q], nparts = grp_start[q + 1] - grp_start[q];
  const int b = jb.order[first + q];
  const int n = jb.n[b];
  double* sig = reinterpret_cast<double*>(smem);                 // scales, then the pair parameters
  RotParams* rp = reinterpret_cast<RotParams*>(smem + jacobi_scale_bytes(n));
  double* wsA = jb.ws + jb.ws_off[b];
  double* wsV = wsA + (size_t)n * n * 2;
  Mat<false> A{reinterpret_cast<c64*>(wsA), n}, V{reinterpret_cast<c64*>(wsV), n};
  jacobi_problem<false, 2, WA>(n, jb.A + jb.a_off[b] * 2 * WA, A, V, rp, sig, jb.red + (size_t)q * red_stride, jb.max_sweeps,
                               jb.flops, jb.W + jb.w_off[b], jb.V + jb.a_off[b] * 2, jb.info + b, part, nparts, gb + q);
}

size_t jacobi_smem_bytes(int n) {
  return (size_t)2 * (n + 1) * n * sizeof(c64) + (size_t)(n / 2 + 1) * sizeof(RotParams) + (size_t)n * sizeof(double);
}

template <int WA>
static zkq_status launch_words(const JacobiBatch& jb, int n_small, int n_large, int max_small_n, int max_large_n,
                               int cluster, int grid_blocks, GridBar* gb, const int32_t* grp_start, int red_stride,
                               cudaStream_t st) {
  if (n_small > 0) {
    size_t sm = jacobi_smem_bytes(max_small_n);
    ZKQ_CUDA_TRY(smem_limit_max<jacobi_smem_kernel<WA>>());
    ProfScope ps(jb.prof_class, st);
    jacobi_smem_kernel<WA><<<n_small, 256, sm, st>>>(jb, 0, n_small);
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  if (n_large > 0 && grid_blocks > 0) {
    size_t sm = jacobi_scale_bytes(max_large_n) + (size_t)(max_large_n / 2 + 1) * sizeof(RotParams);
    ZKQ_CUDA_TRY(smem_limit_max<jacobi_grid_kernel<WA>>());
    ZKQ_CUDA_TRY(cudaMemsetAsync(gb, 0, sizeof(GridBar) * n_large, st));
    JacobiBatch jbc = jb;
    int first = n_small, count = n_large;
    void* args[] = {&jbc, &first, &count, &gb, &grp_start, &red_stride};
    ProfScope ps(jb.prof_class, st);
    ZKQ_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)jacobi_grid_kernel<WA>, dim3(grid_blocks), dim3(256), args, sm, st));
    return ZKQ_OK;
  }
  if (n_large > 0) {
    size_t sm = jacobi_scale_bytes(max_large_n) + (size_t)2 * (max_large_n / 2 + 1) * sizeof(RotParams);   // scales, pairs, staging share
    ZKQ_CUDA_TRY(smem_limit_max<jacobi_global_kernel<WA>>());
    if (cluster > 8)
      ZKQ_CUDA_TRY(cudaFuncSetAttribute(jacobi_global_kernel<WA>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_large * cluster);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr; cfg.numAttrs = 1;
    ProfScope ps(jb.prof_class, st);
    ZKQ_CUDA_TRY(cudaLaunchKernelEx(&cfg, jacobi_global_kernel<WA>, jb, n_small));
  }
  return ZKQ_OK;
}

zkq_status launch_jacobi(const JacobiBatch& jb, int a_words, int n_small, int n_large, int max_small_n,
                         int max_large_n, int cluster, int grid_blocks, GridBar* gb, const int32_t* grp_start,
                         int red_stride, cudaStream_t st) {
  switch (a_words) {
    case 1: return launch_words<1>(jb, n_small, n_large, max_small_n, max_large_n, cluster, grid_blocks, gb, grp_start, red_stride, st);
    case 2: return launch_words<2>(jb, n_small, n_large, max_small_n, max_large_n, cluster, grid_blocks, gb, grp_start, red_stride, st);
    case 4: return launch_words<4>(jb, n_small, n_large, max_small_n, max_large_n, cluster, grid_blocks, gb, grp_start, red_stride, st);
    default: return ZKQ_EINVAL;
  }
}

zkq_status set_grid_barrier_hook(int extra_arrivals, int log2_poll_limit) {
  if (extra_arrivals < 0 || extra_arrivals > 1 || log2_poll_limit < 4 || log2_poll_limit > 22) return ZKQ_EINVAL;
  const WaitHook h{extra_arrivals, log2_poll_limit};
  ZKQ_CUDA_TRY(cudaMemcpyToSymbol(g_wait_hook, &h, sizeof(h)));
  return ZKQ_OK;
}

int jacobi_grid_max_blocks(int max_large_n, int a_words) {
  size_t sm = jacobi_scale_bytes(max_large_n) + (size_t)(max_large_n / 2 + 1) * sizeof(RotParams);
  int per_sm = 0;
  cudaError_t e = cudaSuccess;
  if (a_words == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_grid_kernel<1>, 256, sm);
  else if (a_words == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_grid_kernel<2>, 256, sm);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_grid_kernel<4>, 256, sm);
  if (e != cudaSuccess) { set_last_cuda_error(e); return 0; }
  return per_sm;
}

}  // namespace zkq
