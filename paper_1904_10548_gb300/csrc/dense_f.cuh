// The shared operator F applied as a dense matrix, for a dense W_u.
//
// With W_u not diagonal the sparse Schur form of F = W^-1 - W^-1 E' S^-1 E
// W^-1 no longer holds, but F is still one matrix shared by every node of
// the tree (the collapse of the per-node recursion of paper §4.4 does not
// depend on W_u being diagonal).  z_q = F ghat_q / (2 p_q) for the m rows of
// a chain segment or a group is then a product of the stacked ghat rows
// (m x nu) with F (nu x nu):
//   FP64 (the FP64 kernel and the FP64 steps of the mixed kernel): each
//     thread forms its components for a block of rows with FMAs, F read
//     column by column from L2 (F symmetric, so a column is a row);
//   FP32 (the iterations of the mixed kernel): tensor cores, one warp-level
//     mma.m16n8k8 of TF32 per 16 rows x 8 columns x 8 terms, each operand
//     split into a TF32 head and a TF32 tail so that head*head + head*tail +
//     tail*head carries about as many bits as an FP32 product (the split
//     product of Markidis et al. 2018 and Ootomo & Yokota 2022), accumulated
//     in FP32.  F's fragments are laid out on the host in the order the warps
//     load them (dense_f_fragments in rapidnet.cu).
// Both write z over ghat in place, so every row is read in full before the
// team's barrier and written after it.
#pragma once

#include "kernels.cuh"

// Team, Map2 and map2 come from solve_device.cuh, which includes this file.

namespace rn {

// TF32 head of an FP32 value (round to nearest, ties away), as its bits
__device__ __forceinline__ unsigned tf32_head(float a) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
  return r;
}

// D += A B for one 16 x 8 x 8 TF32 tile (FP32 accumulators)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// FP64: z = F ghat / (2p) for m rows, in place, in blocks of RPT rows per
// thread; JC components per thread (the team's width is at least nu / 2)
template <int RPT, int JC, typename RowF>
__device__ void dense_rows(const NetDev<double> &nt, int m, RowF row, const double *i2p,
                           const Team &tm, const Map2 &mp) {
  const int nu = nt.nu, NXP = nt.NXP;
  const double *F = nt.Fd;
  for (int q0 = 0; q0 < m; q0 += RPT * mp.rs) {
    double acc[JC][RPT];
#pragma unroll
    for (int jj = 0; jj < JC; ++jj)
#pragma unroll
      for (int r = 0; r < RPT; ++r) acc[jj][r] = 0.0;
    for (int k = 0; k < nu; ++k) {
      double gv[RPT];
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int q = q0 + mp.r0 + r * mp.rs;
        gv[r] = q < m ? row(q)[NXP + k] : 0.0;
      }
#pragma unroll
      for (int jj = 0; jj < JC; ++jj) {
        const int j = mp.c0 + jj * mp.cw;
        if (j < nu) {
          const double f = __ldg(F + (size_t)k * nu + j);  // F[k][j] = F[j][k]
#pragma unroll
          for (int r = 0; r < RPT; ++r) acc[jj][r] += f * gv[r];
        }
      }
    }
    tm.sync();
#pragma unroll
    for (int jj = 0; jj < JC; ++jj) {
      const int j = mp.c0 + jj * mp.cw;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int q = q0 + mp.r0 + r * mp.rs;
        if (j < nu && q < m) row(q)[NXP + j] = acc[jj][r] * i2p[q];
      }
    }
    tm.sync();
  }
}

template <typename RowF>
__device__ void apply_F_dense(const NetDev<double> &nt, int m, RowF row, const double *i2p,
                              const Team &tm) {
  const Map2 mp = map2(tm, nt.nu);
  if (nt.nu <= mp.cw)
    dense_rows<8, 1>(nt, m, row, i2p, tm, mp);
  else
    dense_rows<4, 2>(nt, m, row, i2p, tm, mp);
}

// FP32 on tensor cores: z = F ghat / (2p) for m rows, in place.  Warp w of
// the team takes the n-tiles w, w + nw, ... (at most kTcTiles of them) for
// each block of 16 rows; Ft holds per (k-step, n-tile, lane) the B
// fragment {b0, b1} of F as TF32 heads and tails.
template <typename RowF>
__device__ void apply_F_tc(const NetDev<float> &nt, int m, RowF row, const float *i2p,
                           const Team &tm) {
  const int nu = nt.nu, NXP = nt.NXP;
  const int NT = (nu + 7) >> 3;  // n-tiles = k-steps
  const int lane = tm.lane(), warp = tm.warp(), nw = tm.nwarps();
  const int g = lane >> 2, t = lane & 3;
  const float4 *Ft = nt.Ft;
  for (int q0 = 0; q0 < m; q0 += 16) {
    const int qa = q0 + g, qb = q0 + g + 8;
    const float *ra = qa < m ? row(qa) + NXP : nullptr;
    const float *rb = qb < m ? row(qb) + NXP : nullptr;
    float acc[kTcTiles][4];
#pragma unroll
    for (int i = 0; i < kTcTiles; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    for (int ks = 0; ks < NT; ++ks) {
      const int k0 = 8 * ks + t, k1 = k0 + 4;
      const float av[4] = {(ra && k0 < nu) ? ra[k0] : 0.f, (rb && k0 < nu) ? rb[k0] : 0.f,
                           (ra && k1 < nu) ? ra[k1] : 0.f, (rb && k1 < nu) ? rb[k1] : 0.f};
      unsigned ah[4], al[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        ah[e] = tf32_head(av[e]);
        al[e] = tf32_head(av[e] - __uint_as_float(ah[e]));
      }
#pragma unroll
      for (int i = 0; i < kTcTiles; ++i) {
        const int nt_ = warp + i * nw;
        if (nt_ < NT) {
          const float4 b = __ldg(Ft + ((size_t)ks * NT + nt_) * 32 + lane);
          const unsigned bh0 = __float_as_uint(b.x), bh1 = __float_as_uint(b.y);
          const unsigned bl0 = __float_as_uint(b.z), bl1 = __float_as_uint(b.w);
          mma_tf32(acc[i], al, bh0, bh1);
          mma_tf32(acc[i], ah, bl0, bl1);
          mma_tf32(acc[i], ah, bh0, bh1);
        }
      }
    }
    tm.sync();
#pragma unroll
    for (int i = 0; i < kTcTiles; ++i) {
      const int nt_ = warp + i * nw;
      const int c0 = 8 * nt_ + 2 * t;
      if (nt_ < NT) {
        if (qa < m) {
          float *z = row(qa) + NXP;
          if (c0 < nu) z[c0] = acc[i][0] * i2p[qa];
          if (c0 + 1 < nu) z[c0 + 1] = acc[i][1] * i2p[qa];
        }
        if (qb < m) {
          float *z = row(qb) + NXP;
          if (c0 < nu) z[c0] = acc[i][2] * i2p[qb];
          if (c0 + 1 < nu) z[c0 + 1] = acc[i][3] * i2p[qb];
        }
      }
    }
    tm.sync();
  }
}

}  // namespace rn
