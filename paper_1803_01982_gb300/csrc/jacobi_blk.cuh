// jacobi_blk.cuh -- SVD of the small k x k factor M of tmp = Q_t M (Alg. 9,
// "svd(tmp)") in single precision: one-sided (Hestenes) Jacobi on X = M^T
// with whole columns distributed in blocks over a thread-block cluster.
//
//   X J = W diag(sigma) with J orthogonal (started at I, accumulating the
//   rotations), so M = J diag(sigma) W^T: U_s = J, V_s = W = the columns of
//   the rotated X normalised, sigma_c = ||x_c||.
//
// Layout.  The k columns (padded with zero columns to kp = 2 C b) form 2C
// blocks of b columns; each of the C blocks of the cluster holds two of them
// ("slots"), every column whole: its k rows of X and its k rows of J, in
// shared memory.  So the three dot products of a pair are local to one block
// and need no exchange between blocks.
//
// Ordering of one sweep (every pair of columns meets exactly once):
//   1. intra rounds: the pairs inside each block, a round-robin among the b
//      columns of a block (with a bye when b is odd), both blocks of every
//      block of the cluster at once;
//   2. 2C - 1 outer rounds over the blocks by the circle method (block 2C-1
//      fixed in block 0, the others moving one position per round); in outer
//      round t the two blocks held by a cluster block meet in b inner rounds,
//      inner round r pairing column q of slot 0 with column (q + r) mod b of
//      slot 1.  Pair slot q keeps column q of slot 0 in registers for the
//      whole outer round; the slot-1 columns stay in shared memory.
//   Between outer rounds each block pushes its two blocks into the second
//   buffers of the blocks that hold them next (bulk copies into distributed
//   shared memory, completing on the receivers' mbarriers), after one
//   cluster barrier.  A pair costs half a warp:
//   its 16 lanes hold the row pairs 32 e + 2 g + {0, 1} (one 8-byte shared
//   memory access per pair of rows, consecutive across lanes), the dot
//   products are 16-lane sums, so each shuffle serves the two pairs of a
//   warp.
//
// Accuracy.  The rotation (Rutishauser's formulas, single precision) is
// orthogonal only to rounding, and in single precision that rounding drifts
// the column norms of J and X together by about 1e-5 over the ~2000
// rotations a column takes.  Since X = X_0 J exactly up to the rounding of
// each application, a column norm drift of J is the same factor in X, so
// sigma_c = ||x_c|| / ||j_c|| and the normalised columns of J and X remove
// it: on the 20000 x 20000 benchmark factors this brings the singular values
// from 2e-5 to 1e-6 relative of the FP64 SVD and both factors to
// orthonormality 1e-6 .. 3e-6.  The norms are accumulated in FP64.
//
// Convergence: a pair is rotated when |x_p . x_q| > tol ||x_p|| ||x_q||; the
// sweeps end after a sweep without rotations, decided from the rotation
// counts of all blocks (read through distributed shared memory after a
// cluster barrier, so every block takes the same decision).  There are no
// spin waits: the only waits are block and cluster barriers, which every
// block of the cluster reaches in the same sequence.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace ffq {

constexpr int JB_G = 16;         // lanes per pair (a warp holds two pairs)
constexpr int JB_MAX_NE = 7;    // row pairs per lane (k <= 224 = 32 * 7)
constexpr int JB_MAX_B = 14;    // columns per block (2 C b >= k with C = 8)
constexpr int JB_MAX_SWEEPS = 40;

struct JbGeom {
  int C, b, kp, ne, kr, cs, nw;  // blocks of the cluster, block width, padded columns, row pairs per lane,
                                 // padded rows, column stride (floats: X rows then J rows), warps
};

__host__ __device__ inline JbGeom jb_geom(int k, int C) {
  JbGeom g;
  g.C = C;
  g.b = (k + 2 * C - 1) / (2 * C);
  g.kp = 2 * C * g.b;
  g.ne = (k + 2 * JB_G - 1) / (2 * JB_G);
  g.kr = 2 * JB_G * g.ne;
  g.cs = 2 * g.kr;
  g.nw = (g.b + 1) / 2;  // two pairs per warp: b cross pairs, <= b intra pairs
  return g;
}

// Cluster size for a given k: enough blocks that b <= JB_MAX_B, few enough
// that each has work.
__host__ __device__ inline int jb_cluster_for(int k) { return k > 64 ? 8 : (k > 16 ? 4 : 2); }

inline size_t jb_smem_bytes(int k) {
  const JbGeom g = jb_geom(k, jb_cluster_for(k));
  return (size_t)2 * 2 * g.b * g.cs * sizeof(float)  // two buffers of two slots
         + (size_t)2 * g.b * (sizeof(float) + sizeof(int) + 2 * sizeof(double)) + 64;
}

// Block of the circle method held in (cluster block c, slot) at outer round t.
__device__ __forceinline__ int jb_block_of(int c, int slot, int t, int C) {
  const int n1 = 2 * C - 1;
  if (c == 0) return slot == 0 ? n1 : t;
  return slot == 0 ? (t + c) % n1 : (t - c + n1) % n1;
}

// Where block x is at outer round t.
__device__ __forceinline__ void jb_owner(int x, int t, int C, int &c, int &slot) {
  const int n1 = 2 * C - 1;
  if (x == n1) {
    c = 0;
    slot = 0;
    return;
  }
  const int d = (x - t + n1) % n1;
  if (d == 0) {
    c = 0;
    slot = 1;
  } else if (d <= C - 1) {
    c = d;
    slot = 0;
  } else {
    c = n1 - d;
    slot = 1;
  }
}

// Sum over the 16 lanes of a half warp (both halves at once).
__device__ __forceinline__ float jb_sum16(float v) {
#pragma unroll
  for (int o = JB_G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Rotation (cs, sn) that makes a pair orthogonal (Rutishauser's formulas),
// none (sn = 0) when |ga| <= tol sqrt(al be): zeta = (be - al) / (2 ga),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) (the smaller angle, |t| <= 1),
// cs = 1 / sqrt(1 + t^2) refined by one Newton step so that cs^2 + sn^2 = 1
// to rounding, sn = cs t.
__device__ __forceinline__ void jb_rotation(float al, float be, float ga, float tol, float &cs, float &sn,
                                            float &tn) {
  cs = 1.f;
  sn = 0.f;
  tn = 0.f;
  if (!(ga != 0.f && ga * ga > (tol * tol) * (al * be))) return;
  const float zeta = __fdividef(be - al, 2.f * ga);
  const float a = fabsf(zeta);
  float root = a;  // sqrt(1 + a^2), = a to rounding for a >= 2^30
  if (a < 1073741824.f) {
    const float x = fmaf(a, a, 1.f);
    root = x * rsqrtf(x);
  }
  const float t = copysignf(__fdividef(1.f, a + root), zeta);
  const float x = fmaf(t, t, 1.f);
  float y = rsqrtf(x);
  y = y * fmaf(-0.5f * x, y * y, 1.5f);
  cs = y;
  sn = y * t;
  tn = t;
}

// The three dot products of a pair over the lane's row pairs, summed over
// the pair's 16 lanes (two accumulators each, to halve the FMA chains).
__device__ __forceinline__ void jb_dots(const float2 *ax, const float2 *bx, float &al, float &be, float &ga) {
  float2 a2[2], b2[2], g2[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) a2[h] = b2[h] = g2[h] = make_float2(0.f, 0.f);
#pragma unroll
  for (int e = 0; e < JB_MAX_NE; ++e) {
    a2[e & 1] = __ffma2_rn(ax[e], ax[e], a2[e & 1]);
    b2[e & 1] = __ffma2_rn(bx[e], bx[e], b2[e & 1]);
    g2[e & 1] = __ffma2_rn(ax[e], bx[e], g2[e & 1]);
  }
  al = jb_sum16((a2[0].x + a2[1].x) + (a2[0].y + a2[1].y));
  be = jb_sum16((b2[0].x + b2[1].x) + (b2[0].y + b2[1].y));
  ga = jb_sum16((g2[0].x + g2[1].x) + (g2[0].y + g2[1].y));
}

// (a, b) <- (cs a - sn b, sn a + cs b) on the lane's row pairs.
__device__ __forceinline__ void jb_rotate(float2 *a, float2 *b, float cs, float sn) {
  const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), n2 = make_float2(-sn, -sn);
#pragma unroll
  for (int e = 0; e < JB_MAX_NE; ++e) {
    const float2 x0 = a[e], y0 = b[e];
    a[e] = __ffma2_rn(c2, x0, __fmul2_rn(n2, y0));
    b[e] = __ffma2_rn(s2, x0, __fmul2_rn(c2, y0));
  }
}

// Column (X rows then J rows, stride kr between the parts) to registers:
// lane g of the pair holds rows 32 e + 2 g + {0, 1}; row pairs past the
// column's ne groups read as zero.
__device__ __forceinline__ void jb_load(const float *col, int kr, int ne, int g, float2 *x, float2 *j) {
#pragma unroll
  for (int e = 0; e < JB_MAX_NE; ++e) {
    x[e] = (e < ne) ? *reinterpret_cast<const float2 *>(col + 2 * g + 2 * JB_G * e) : make_float2(0.f, 0.f);
    j[e] = (e < ne) ? *reinterpret_cast<const float2 *>(col + kr + 2 * g + 2 * JB_G * e) : make_float2(0.f, 0.f);
  }
}
__device__ __forceinline__ void jb_store(float *col, int kr, int ne, int g, const float2 *x, const float2 *j) {
#pragma unroll
  for (int e = 0; e < JB_MAX_NE; ++e)
    if (e < ne) {
      *reinterpret_cast<float2 *>(col + 2 * g + 2 * JB_G * e) = x[e];
      *reinterpret_cast<float2 *>(col + kr + 2 * g + 2 * JB_G * e) = j[e];
    }
}

// Block exchange between outer rounds: each block pushes its two column
// blocks into the blocks that hold them next, with bulk copies from its own
// shared memory into theirs (the async proxy), each completing on the
// receiver's mbarrier.  The receiver arms that barrier for the two blocks it
// will receive before the cluster barrier that ends the round, so the arming
// precedes every push; every wait is bounded (~1 s) and flags a timeout.
constexpr long long JB_SPIN = 4000000;

__device__ __forceinline__ uint32_t jb_smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t jb_mapa(uint32_t addr, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void jb_mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(jb_smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void jb_mbar_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(jb_smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool jb_mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(jb_smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// A wait gives up after ~1 s of wall time (or JB_SPIN polls), or at once when
// a timeout was already flagged, so that a failed exchange ends the kernel in
// seconds with STATUS_TIMEOUT rather than one second per remaining round.
__device__ __forceinline__ void jb_mbar_wait(uint64_t *bar, uint32_t parity, int *ctl) {
  if (jb_mbar_try(bar, parity)) return;
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  long long spins = 0;
  while (!jb_mbar_try(bar, parity)) {
    if ((++spins & 255) == 0) {
      unsigned long long t1;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
      if (*((volatile int *)(ctl + CTL_TIMEOUT)) != 0 || t1 - t0 > 1000000000ull || spins > JB_SPIN) {
        atomicExch(ctl + CTL_TIMEOUT, 1);
        set_status(ctl, STATUS_TIMEOUT);
        return;
      }
    }
  }
}
// bytes (a multiple of 16) from this block's shared memory at src to the
// cluster-shared address dst, completing on the cluster-shared mbarrier bar.
__device__ __forceinline__ void jb_push(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "r"(jb_smem_addr(src)), "r"(bytes), "r"(bar)
      : "memory");
}

// M (k x k, row-major, leading dimension ldm) -> Uout = U_s, Vout = V_s
// (k x k, row-major, leading dimension k), Sout (k, descending).  Cluster of
// C = jb_cluster_for(k) blocks of 32 * jb_geom(k, C).nw threads.
__device__ __forceinline__ void jacobi_blk_body(const float *__restrict__ M, int k, int ldm, float tol,
                                                int max_sweeps, float *__restrict__ Uout,
                                                float *__restrict__ Sout, float *__restrict__ Vout, int *ctl) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int c = (int)cluster.block_rank();
  const JbGeom geo = jb_geom(k, C);
  const int b = geo.b, ne = geo.ne, kr = geo.kr, cs = geo.cs, n1 = 2 * C - 1;
  extern __shared__ __align__(16) float jb_sm[];
  const int bufsz = 2 * b * cs;                              // floats of one buffer (two slots)
  float *sig = jb_sm + 2 * bufsz;                            // [2b]
  int *gid = reinterpret_cast<int *>(sig + 2 * b);           // [2b]
  double *xnr = reinterpret_cast<double *>(                  // [2b] ||x||, then [2b] ||j||
      (reinterpret_cast<uintptr_t>(gid + 2 * b) + 7) & ~(uintptr_t)7);
  double *jnr = xnr + 2 * b;
  __shared__ int s_cnt[2];
  __shared__ __align__(8) uint64_t s_bar;  // arrival of the next outer round's two blocks
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int q = 2 * w + (lane >> 4);  // pair slot of this half warp
  const int g = lane & (JB_G - 1);    // lane within the pair
  if (max_sweeps > JB_MAX_SWEEPS) max_sweeps = JB_MAX_SWEEPS;

  // the two blocks of outer round 0: X(:, gc) = row gc of M, J = I
  for (int s = 0; s < 2; ++s) {
    const int x = jb_block_of(c, s, 0, C);
    for (int e = threadIdx.x; e < b * kr; e += blockDim.x) {
      const int i = e / kr, r = e - i * kr, gc = x * b + i;
      float *col = jb_sm + (s * b + i) * cs;
      col[r] = (gc < k && r < k) ? M[(size_t)gc * ldm + r] : 0.f;
      col[kr + r] = (gc < k && r == gc) ? 1.f : 0.f;
    }
  }
  if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) jb_mbar_init(&s_bar);
  __syncthreads();
  cluster.sync();
  const uint32_t slot_bytes = (uint32_t)(b * cs * sizeof(float));
  uint32_t bar_phase = 0;

  const int ph = b / 2;                     // pairs per block in an intra round
  const int nb = b + (b & 1), m1 = nb - 1;  // players of the intra round-robin (with a bye if b is odd)
  int cur = 0, tpos = 0, sweeps = 0;
  bool done = false;
  while (sweeps < max_sweeps && !done) {
    int nrot = 0;  // rotations counted on lane 0 of each pair
    if (threadIdx.x == 0) s_cnt[sweeps & 1] = 0;
    __syncthreads();
    float *B = jb_sm + cur * bufsz;
    // 1. intra rounds (positions of outer round 0)
    if (ph > 0) {
      for (int t = 0; t < m1; ++t) {
        const bool on = q < 2 * ph;
        float2 px[JB_MAX_NE], pj[JB_MAX_NE], qx[JB_MAX_NE], qj[JB_MAX_NE];
        float *cp = B, *cq = B;
        if (on) {
          const int sl = q / ph, i = q % ph + (b & 1);  // odd b: pair 0 holds the bye
          int p0, q0;
          if (i == 0) {
            p0 = t;
            q0 = m1;
          } else {
            p0 = (t + i) % m1;
            q0 = (t - i + m1) % m1;
          }
          cp = B + (sl * b + p0) * cs;
          cq = B + (sl * b + q0) * cs;
        }
        jb_load(cp, kr, on ? ne : 0, g, px, pj);
        jb_load(cq, kr, on ? ne : 0, g, qx, qj);
        float al, be, ga, c_, s_, t_;
        jb_dots(px, qx, al, be, ga);
        jb_rotation(al, be, ga, tol, c_, s_, t_);
        if (on && s_ != 0.f) {
          jb_rotate(px, qx, c_, s_);
          jb_rotate(pj, qj, c_, s_);
          jb_store(cp, kr, ne, g, px, pj);
          jb_store(cq, kr, ne, g, qx, qj);
          nrot += (g == 0);
        }
        __syncthreads();
      }
    }
    // 2. outer rounds over the blocks
    for (int t = 0; t < n1; ++t) {
      const bool on = q < b;
      float2 ax[JB_MAX_NE], aj[JB_MAX_NE];
      float *ca = B + (on ? q : 0) * cs;
      jb_load(ca, kr, on ? ne : 0, g, ax, aj);
      int jc = on ? q : 0;  // slot-1 column of inner round r: (q + r) mod b
      for (int r = 0; r < b; ++r) {
        float *cb = B + (b + jc) * cs;
        float2 bx[JB_MAX_NE], bj[JB_MAX_NE];
        jb_load(cb, kr, on ? ne : 0, g, bx, bj);
        float al, be, ga, c_, s_, t_;
        jb_dots(ax, bx, al, be, ga);
        jb_rotation(al, be, ga, tol, c_, s_, t_);
        if (on && s_ != 0.f) {
          jb_rotate(ax, bx, c_, s_);
          jb_rotate(aj, bj, c_, s_);
          jb_store(cb, kr, ne, g, bx, bj);
          nrot += (g == 0);
        }
        jc = (jc + 1 == b) ? 0 : jc + 1;
        __syncthreads();
      }
      if (on) jb_store(ca, kr, ne, g, ax, aj);
      const bool last = (t == n1 - 1);
      if (last && nrot) atomicAdd(&s_cnt[sweeps & 1], nrot);
      if (threadIdx.x == 0) jb_mbar_expect(&s_bar, 2 * slot_bytes);  // this round's two incoming blocks
      cluster.sync();  // every block's round-t blocks (and counts) are final; every barrier is armed
      if (last) {
        int tot = 0;
        for (int cc = 0; cc < C; ++cc) tot += *cluster.map_shared_rank(&s_cnt[sweeps & 1], (unsigned)cc);
        if (c == 0 && threadIdx.x == 0 && sweeps < 16) ctl[CTL_SWEEP_ROT0 + sweeps] = tot;
        done = (tot == 0);
        if (done) break;  // the blocks stay where outer round t left them
      }
      // push this block's two blocks to the blocks that hold them in the next
      // outer round (into their other buffer), then wait for the two coming in
      const int tn = last ? 0 : t + 1;
      float *Bn = jb_sm + (cur ^ 1) * bufsz;
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int s = 0; s < 2; ++s) {
          int dc, ds;
          jb_owner(jb_block_of(c, s, t, C), tn, C, dc, ds);
          jb_push(jb_mapa(jb_smem_addr(Bn + ds * b * cs), (unsigned)dc), B + s * b * cs, slot_bytes,
                  jb_mapa(jb_smem_addr(&s_bar), (unsigned)dc));
        }
      }
      jb_mbar_wait(&s_bar, bar_phase, ctl);
      bar_phase ^= 1;
      cur ^= 1;
      B = Bn;
      tpos = tn;
      if (last) nrot = 0;
    }
    ++sweeps;
  }
  if (c == 0 && threadIdx.x == 0) ctl[CTL_JACOBI_SWEEPS] = sweeps;

  // outputs: sigma_c = ||x_c|| / ||j_c|| (FP64 sums), ranked in descending order
  const float *B = jb_sm + cur * bufsz;
  for (int lc = w; lc < 2 * b; lc += nw) {
    const float *col = B + (size_t)lc * cs;
    double xs = 0.0, js = 0.0;
    for (int r = lane; r < kr; r += 32) {
      const double x = col[r], y = col[kr + r];
      xs = fma(x, x, xs);
      js = fma(y, y, js);
    }
    xs = warp_sum(xs);
    js = warp_sum(js);
    if (lane == 0) {
      const int gc = jb_block_of(c, lc / b, tpos, C) * b + lc % b;
      xnr[lc] = sqrt(xs);
      jnr[lc] = sqrt(js);
      gid[lc] = gc;
      sig[lc] = (gc < k) ? (float)((js > 0.0) ? sqrt(xs) / sqrt(js) : 0.0) : -1.f;
    }
  }
  cluster.sync();
  for (int lc = w; lc < 2 * b; lc += nw) {
    const int gc = gid[lc];
    if (gc >= k) continue;
    const float sc = sig[lc];
    int rk = 0;
    for (int cc = 0; cc < C; ++cc) {
      const float *rs = cluster.map_shared_rank(sig, (unsigned)cc);
      const int *ri = cluster.map_shared_rank(gid, (unsigned)cc);
      for (int e = lane; e < 2 * b; e += 32) {
        const int gd = ri[e];
        if (gd < k) {
          const float sd = rs[e];
          rk += (sd > sc) || (sd == sc && gd < gc);
        }
      }
    }
    rk = warp_sum(rk);
    const float *col = B + (size_t)lc * cs;
    const double xn = xnr[lc], jn = jnr[lc];
    const float ix = (xn > 0.0) ? (float)(1.0 / xn) : 0.f, ij = (jn > 0.0) ? (float)(1.0 / jn) : 0.f;
    for (int r = lane; r < k; r += 32) {
      Uout[(size_t)r * k + rk] = col[kr + r] * ij;
      Vout[(size_t)r * k + rk] = (xn > 0.0) ? col[r] * ix : ((r == rk) ? 1.f : 0.f);
    }
    if (lane == 0) Sout[rk] = sc;
  }
  cluster.sync();  // no block leaves while another may still read its sigma and ids
}

__global__ void __launch_bounds__(32 * ((JB_MAX_B + 1) / 2)) jacobi_blk_kernel(
    const float *__restrict__ M, int k, int ldm, float tol, int max_sweeps, float *__restrict__ Uout,
    float *__restrict__ Sout, float *__restrict__ Vout, int *ctl) {
  jacobi_blk_body(M, k, ldm, tol, max_sweeps, Uout, Sout, Vout, ctl);
}

// Several problems' small SVDs in one launch: cluster i (blocks
// i C .. i C + C - 1) runs problem i exactly as jacobi_blk_kernel would (the
// same cluster size C for all of them, blockDim the largest any of them
// needs: warps past a problem's own need take no pair), so every result is
// bitwise the one a launch of its own gives.
struct JbProblem {
  const float *M;
  float *U, *S, *V;
  int *ctl;
  int k, ldm;
  float tol;
};
constexpr int JB_BATCH_MAX = 32;  // problems per launch (the descriptors travel as kernel parameters)
struct JbBatch {
  int count, max_sweeps;
  JbProblem p[JB_BATCH_MAX];
};

__global__ void __launch_bounds__(32 * ((JB_MAX_B + 1) / 2)) jacobi_blk_batch_kernel(const JbBatch batch) {
  namespace cg = cooperative_groups;
  const int i = (int)(blockIdx.x / cg::this_cluster().num_blocks());
  const JbProblem &q = batch.p[i];
  jacobi_blk_body(q.M, q.k, q.ldm, q.tol, batch.max_sweeps, q.U, q.S, q.V, q.ctl);
}

}  // namespace ffq
