// dmr_adjoint.cuh -- hand-written reverse-mode (adjoint) kernels of the DMR
// time step with the refinement schedule held fixed.
//
// Each forward operation of dmr_kernels.cuh is transposed in gather form
// where every output has one writer (no atomics), and scatter form with
// atomics where several fine samples map to one coarse sample (Eq. 5a/5b
// transposes).  Notation: a* is the adjoint (dL/d*) of a forward variable.
//
// Forward EM step at level l (see k_em), per mesh:
//   S2 += e2(E^l)                       (if the level is an E^2 sample)
//   H'  = H - ch curlE(E^l)
//   v'  = va v - vb (E^l + inc)
//   E'  = E^l + ce curlH(H') + cj (n_a + n_b) v'          interior edges
//   E'_b = E^l_1 + mur (E'_1 - E^l_b)                      Mur sides
//   E'_b = Eq. 5b(coarse E^n, coarse E^{n+1})              coarse-fine sides
// Reverse: Mur^T, Eq. 5b^T (scatter to coarse), E^T, v^T, H^T, S2^T.
#pragma once
#include "dmr_kernels.cuh"

namespace dmr {

// Tape copies of a recorded step in one launch: job q copies n16[q] 16-byte
// words from src[q] to dst[q] (blockIdx.y = job, grid-stride along x).
constexpr int kTapeJobs = 16;
struct TapeJobs {
  const int4* src[kTapeJobs];
  int4* dst[kTapeJobs];
  long long n16[kTapeJobs];
  int n;
};

__global__ void ka_tape_gather(TapeJobs J) {
  const int q = blockIdx.y;
  if (q >= J.n) return;
  const int4* __restrict__ s = J.src[q];
  int4* __restrict__ d = J.dst[q];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < J.n16[q]; k += stride) d[k] = s[k];
}

template <class T>
struct AdjM {
  const T *aEx_in, *aEy_in;   // adjoint of E^{l+1}
  T *aEx_out, *aEy_out;       // adjoint of E^l (accumulated with +=)
  const T* aHz;               // adjoint of H^{l+1/2} (ka_eh: before the step's own curl share)
  T* aHz_out;                 // ka_eh: adjoint of H^{l-1/2} (the other buffer of the pair)
  T *avx, *avy;               // adjoint of v^{l+1/2} in, of v^{l-1/2} out (in place)
  T* an;                      // adjoint of n (accumulated)
  const T* aS2;               // adjoint of the period's S2 sum (nodes)
  int nx, ny, p;
};

template <class T>
struct FwdM {                 // recorded forward values of the step
  const T *Ex, *Ey;           // E^l as the step used it
  const T *vx, *vy;           // v^{l+1/2}
  const T* n;
};

struct Modes { int m[4]; };

template <class T>
__device__ __forceinline__ T adj_x(const AdjM<T>& a, const Modes& md, T mur, int i, int j) {
  // adjoint of interior E'_x(i,j) including what the Mur rows took from it
  const int p = a.p;
  T v = a.aEx_in[j * p + i];
  if (j == 1 && md.m[SIDE_BOTTOM] == BC_MUR) v = v + mur * a.aEx_in[i];
  if (j == a.ny - 1 && md.m[SIDE_TOP] == BC_MUR) v = v + mur * a.aEx_in[a.ny * p + i];
  return v;
}

template <class T>
__device__ __forceinline__ T adj_y(const AdjM<T>& a, const Modes& md, T mur, int i, int j) {
  const int p = a.p;
  T v = a.aEy_in[j * p + i];
  if (i == 1 && md.m[SIDE_LEFT] == BC_MUR) v = v + mur * a.aEy_in[j * p];
  if (i == a.nx - 1 && md.m[SIDE_RIGHT] == BC_MUR) v = v + mur * a.aEy_in[j * p + a.nx];
  return v;
}

// The adjoint of H^{l-1/2} at cell (i, j): that of H^{l+1/2} plus
// ce curlH^T(aE') over the interior edges (after the Mur rows' share).
template <class T>
__device__ __forceinline__ T ka_h_value(const AdjM<T>& a, const Step<T>& c, const Modes& md, int i, int j) {
  T acc = T(0);
  if (j > 0) acc = acc + adj_x(a, md, c.mur, i, j);
  if (j + 1 < a.ny) acc = acc - adj_x(a, md, c.mur, i, j + 1);
  if (i > 0) acc = acc - adj_y(a, md, c.mur, i, j);
  if (i + 1 < a.nx) acc = acc + adj_y(a, md, c.mur, i + 1, j);
  return a.aHz[j * a.p + i] + c.ce * acc;
}

__device__ __forceinline__ double block_sum_d(double v) { return block_sum(v); }

// Coarse side of a reversed coarse step (nullptrs / off on a fine mesh or
// without a rectangle):
//  * the Eq. 5b^T shares of the coarse tangential E^n along the rectangle's
//    coarse-fine sides, gathered by ka_cfb into line buffers (indexed along
//    the line) instead of the edge adjoints: the coarse ka_e adds them to
//    the edges it writes and clears them;
//  * a8^T: the adjoint of a restricted coarse E^n edge goes to its r fine
//    edges (1/r each; the fine E^n adjoint) and the coarse edge keeps 0.
template <class T>
struct CoarseT {
  int side_on[4], side_at[4];   // lines of the coarse-fine sides (row bottom/top, column left/right)
  T* side[4];
  int restr;                     // a8 is transposed at this step
  int I0, J0, I1, J1, r, jlo, jhi, ilo, ihi;
  T *fEx, *fEy;                  // the fine E^n adjoint
  int fp;
};

// Node (i, j) of a reversed EM step: the adjoint of H^{l-1/2} at cell (i, j)
// (from the other H buffer, re-evaluated at the two neighbouring cells the
// edges of the node need), then the gather of aE^l (edges (i, j)), av, an;
// returns the node's E0 share.  The edge adjoints of E^l are stored (the
// output buffer is not cleared before); with a CoarseT the side shares are
// added and a8 transposed.  Every load of a thread comes before its first
// store, so the loads of the in-place arrays (av, an, side lines) and of the
// read-only inputs are all in flight at once.
template <class T>
__device__ __forceinline__ T ka_e_node(const AdjM<T>& a, const FwdM<T>& f, const Step<T>& c, const Modes& md,
                                       const CoarseT<T>& ct, int i, int j) {
  const int nx = a.nx, ny = a.ny, p = a.p;
  T e0 = T(0);
  if (i <= nx && j <= ny) {
    const int id = j * p + i;
    const bool xe = i < nx, ye = j < ny;
    // ---- H adjoints of the cells the node's edges border
    const T h00 = (xe && ye) ? ka_h_value(a, c, md, i, j) : T(0);
    const T h0m = (xe && j > 0) ? ka_h_value(a, c, md, i, j - 1) : T(0);
    const T hm0 = (ye && i > 0) ? ka_h_value(a, c, md, i - 1, j) : T(0);
    // ---- loads: in-place values and side lines
    const T avx0 = xe ? a.avx[id] : T(0);
    const T avy0 = ye ? a.avy[id] : T(0);
    const T an0 = a.an[id];
    const bool s_b = xe && ct.side_on[SIDE_BOTTOM] && j == ct.side_at[SIDE_BOTTOM];
    const bool s_t = xe && ct.side_on[SIDE_TOP] && j == ct.side_at[SIDE_TOP];
    const bool s_l = ye && ct.side_on[SIDE_LEFT] && i == ct.side_at[SIDE_LEFT];
    const bool s_r = ye && ct.side_on[SIDE_RIGHT] && i == ct.side_at[SIDE_RIGHT];
    const T v_b = s_b ? ct.side[SIDE_BOTTOM][i] : T(0);
    const T v_t = s_t ? ct.side[SIDE_TOP][i] : T(0);
    const T v_l = s_l ? ct.side[SIDE_LEFT][j] : T(0);
    const T v_r = s_r ? ct.side[SIDE_RIGHT][j] : T(0);
    T an_acc = T(0);
    // ---- x edge (i, j)
    T outx = T(0), avx1 = T(0);
    if (xe) {
      T out, avt;
      if (j > 0 && j < ny) {
        const T aEa = adj_x(a, md, c.mur, i, j);
        avt = avx0 + c.cj * (f.n[id] + f.n[id + 1]) * aEa;
        out = aEa;
        if (j == 1 && md.m[SIDE_BOTTOM] == BC_MUR) out = out + a.aEx_in[i];
        if (j == ny - 1 && md.m[SIDE_TOP] == BC_MUR) out = out + a.aEx_in[ny * p + i];
        an_acc = an_acc + f.vx[id] * aEa;
      } else {
        const int sd = j == 0 ? SIDE_BOTTOM : SIDE_TOP;
        avt = avx0;
        out = md.m[sd] == BC_MUR ? -c.mur * a.aEx_in[id] : T(0);
      }
      out = out - c.vb * avt;
      T hs = T(0);
      if (j < ny) hs = hs + h00;
      if (j > 0) hs = hs - h0m;
      out = out - c.ch * hs;
      if (c.accum) {
        const T wl = (i > 0) ? T(0.5) : T(1);                 // node i: this is its right edge
        const T wr = (i + 1 < nx) ? T(0.5) : T(1);            // node i+1: its left edge
        out = out + T(2) * f.Ex[id] * (a.aS2[id] * wl + a.aS2[id + 1] * wr);
      }
      avx1 = c.va * avt;
      if (s_b) out = v_b + out;
      if (s_t) out = v_t + out;
      outx = out;
    }
    if (i > 0 && i - 1 < nx && j > 0 && j < ny) an_acc = an_acc + f.vx[id - 1] * adj_x(a, md, c.mur, i - 1, j);
    // ---- y edge (i, j)
    T outy = T(0), avy1 = T(0);
    if (ye) {
      const T phi = c.sphi * c.ckx[i] - c.cphi * c.skx[i];
      T out, avt;
      if (i > 0 && i < nx) {
        const T aEa = adj_y(a, md, c.mur, i, j);
        avt = avy0 + c.cj * (f.n[id] + f.n[id + p]) * aEa;
        out = aEa;
        if (i == 1 && md.m[SIDE_LEFT] == BC_MUR) out = out + a.aEy_in[j * p];
        if (i == nx - 1 && md.m[SIDE_RIGHT] == BC_MUR) out = out + a.aEy_in[j * p + nx];
        an_acc = an_acc + f.vy[id] * aEa;
      } else {
        const int sd = i == 0 ? SIDE_LEFT : SIDE_RIGHT;
        avt = avy0;
        out = md.m[sd] == BC_MUR ? -c.mur * a.aEy_in[id] : T(0);
      }
      out = out - c.vb * avt;
      e0 -= c.vb * avt * phi;
      T hs = T(0);
      if (i < nx) hs = hs - h00;
      if (i > 0) hs = hs + hm0;
      out = out - c.ch * hs;
      if (c.accum) {
        const T ey = f.Ey[id] + c.E0 * phi;
        const T wb = (j > 0) ? T(0.5) : T(1);
        const T wt = (j + 1 < ny) ? T(0.5) : T(1);
        const T g = T(2) * ey * (a.aS2[id] * wb + a.aS2[id + p] * wt);
        out = out + g;
        e0 += g * phi;
      }
      avy1 = c.va * avt;
      if (s_l) out = v_l + out;
      if (s_r) out = v_r + out;
      outy = out;
    }
    if (j > 0 && i > 0 && i < nx) an_acc = an_acc + f.vy[id - p] * adj_y(a, md, c.mur, i, j - 1);
    // ---- stores
    if (xe && ye) a.aHz_out[id] = h00;
    a.an[id] = an0 + c.cj * an_acc;
    if (xe) {
      a.avx[id] = avx1;
      if (s_b) ct.side[SIDE_BOTTOM][i] = T(0);
      if (s_t) ct.side[SIDE_TOP][i] = T(0);
      if (ct.restr && i >= ct.I0 && i < ct.I1 && j >= ct.jlo && j <= ct.jhi) {
        const T t = outx / (T)ct.r;
        T* d = ct.fEx + (size_t)(ct.r * (j - ct.J0)) * ct.fp + ct.r * (i - ct.I0);
        for (int q = 0; q < ct.r; ++q) d[q] += t;
        outx = T(0);
      }
      a.aEx_out[id] = outx;
    }
    if (ye) {
      a.avy[id] = avy1;
      if (s_l) ct.side[SIDE_LEFT][j] = T(0);
      if (s_r) ct.side[SIDE_RIGHT][j] = T(0);
      if (ct.restr && j >= ct.J0 && j < ct.J1 && i >= ct.ilo && i <= ct.ihi) {
        const T t = outy / (T)ct.r;
        T* d = ct.fEy + (size_t)(ct.r * (j - ct.J0)) * ct.fp + ct.r * (i - ct.I0);
        for (int q = 0; q < ct.r; ++q) d[(size_t)q * ct.fp] += t;
        outy = T(0);
      }
      a.aEy_out[id] = outy;
    }
  }
  return e0;
}

// Eq. 5b^T: the adjoint of each coarse-fine boundary edge of the fine mesh goes
// to the coarse tangential E before (old) and after (new) the coarse step.
template <class T>
struct CfbT {
  int mode[4], start[4], len[4], at[4];
  int r;
  T frac;
  T *new_x, *new_y;                   // coarse adjoint arrays of E^{n+1}
  T* old_line[4];                     // E^n shares, per side along its line (CoarseT::side)
  int cp;                             // coarse pitch
};

// Eq. 5b^T of sample q of side SD, if q lies on it; else q is reduced by the
// side's length and false returned.
template <int SD, class T>
__device__ __forceinline__ bool ka_cfb_side(const AdjM<T>& a, const CfbT<T>& b, int& q) {
  if (b.mode[SD] != BC_CFB) return false;
  constexpr bool xs = SD == SIDE_BOTTOM || SD == SIDE_TOP;
  const int nfx = a.nx, nfy = a.ny, p = a.p;
  const int len = xs ? nfx : nfy;
  if (q >= len) { q -= len; return false; }
  T t;
  if (SD == SIDE_BOTTOM) t = a.aEx_in[q];
  else if (SD == SIDE_TOP) t = a.aEx_in[nfy * p + q];
  else if (SD == SIDE_LEFT) t = a.aEy_in[q * p];
  else t = a.aEy_in[q * p + nfx];
  const int num = 2 * q + 1 - b.r, den = 2 * b.r;
  const int fl = (num >= 0) ? num / den : -((-num + den - 1) / den);
  int i0 = b.start[SD] + fl;
  T xp = (T)(num - fl * den) / (T)den;
  if (i0 < 0) { i0 = 0; xp = T(0); }
  if (i0 > b.len[SD] - 2) { i0 = b.len[SD] - 2; xp = T(1); }
  const T one = T(1);
  const T wo0 = (one - b.frac) * (one - xp), wo1 = (one - b.frac) * xp;
  const T wn0 = b.frac * (one - xp), wn1 = b.frac * xp;
  size_t s0, s1;
  T* n;
  if (xs) {
    s0 = (size_t)b.at[SD] * b.cp + i0; s1 = s0 + 1; n = b.new_x;
  } else {
    s0 = (size_t)i0 * b.cp + b.at[SD]; s1 = s0 + b.cp; n = b.new_y;
  }
  atomicAdd(b.old_line[SD] + i0, wo0 * t);
  atomicAdd(b.old_line[SD] + i0 + 1, wo1 * t);
  atomicAdd(n + s0, wn0 * t);
  atomicAdd(n + s1, wn1 * t);
  return true;
}

// Eq. 5b^T of side sample q (the sides in the order bottom, top, left, right)
template <class T>
__device__ __forceinline__ void ka_cfb_sample(const AdjM<T>& a, const CfbT<T>& b, int q) {
  if (ka_cfb_side<SIDE_BOTTOM>(a, b, q)) return;
  if (ka_cfb_side<SIDE_TOP>(a, b, q)) return;
  if (ka_cfb_side<SIDE_LEFT>(a, b, q)) return;
  ka_cfb_side<SIDE_RIGHT>(a, b, q);
}

// A rectangle of node blocks of one mesh in a reversed EM step: blocks
// (bx0 + k % nbx, by0 + k / nbx), each TX x TY nodes, except those inside the
// skip box [sx0, sx1] x [sy0, sy1] (sx0 > sx1: none skipped).
template <class T>
struct NodePart {
  AdjM<T> a;
  FwdM<T> f;
  Step<T> c;
  Modes md;
  CoarseT<T> ct;
  int bx0, by0, nbx, nby;
  int sx0, sx1, sy0, sy1;
};

// Node block k of a part: ka_e_node over its nodes, E0 share summed in FP64.
template <class T>
__device__ __forceinline__ void ka_part_block(const NodePart<T>& P, int k, double* e0acc) {
  const int by = P.by0 + k / P.nbx, bx = P.bx0 + k % P.nbx;
  if (bx >= P.sx0 && bx <= P.sx1 && by >= P.sy0 && by <= P.sy1) return;   // whole block
  const T e0 = ka_e_node(P.a, P.f, P.c, P.md, P.ct, bx * TX + (int)threadIdx.x, by * TY + (int)threadIdx.y);
  const double s = block_sum_d((double)e0);
  if (threadIdx.x == 0 && threadIdx.y == 0 && s != 0.0) atomicAdd(e0acc, s);
}

// One launch of a reversed EM step: the node blocks of part P0 (nb0 blocks),
// then the Eq. 5b^T side samples of P0's fine mesh (ncfb blocks of TX * TY
// samples; they read aE' and add to coarse adjoints only), then the node
// blocks of part P1 (nb1 blocks): coarse nodes away from the rectangle run
// beside the fine sub-steps of the same coarse step, which neither read nor
// write them.
template <class T>
__global__ void __launch_bounds__(TX * TY) ka_eh(NodePart<T> P0, NodePart<T> P1, CfbT<T> cb, int nb0, int ncfb,
                                                 double* e0acc) {
  const int blk = (int)blockIdx.x;
  if (blk < nb0) {
    ka_part_block(P0, blk, e0acc);
  } else if (blk < nb0 + ncfb) {
    ka_cfb_sample(P0.a, cb, (blk - nb0) * TX * TY + (int)(threadIdx.y * TX + threadIdx.x));
  } else {
    ka_part_block(P1, blk - nb0 - ncfb, e0acc);
  }
}

// a8^T for E: the adjoint of a restricted coarse edge goes to its r fine edges
// (1/r each) and is cleared on the coarse mesh.
template <class T>
__global__ void ka_restrict(T* cEx, T* cEy, int cp, T* fEx, T* fEy, int fp, int I0, int J0, int I1,
                            int J1, int r, int jlo, int jhi, int ilo, int ihi) {
  const int i = I0 + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = J0 + blockIdx.y * blockDim.y + threadIdx.y;
  if (i > I1 || j > J1) return;
  const int fa = r * (i - I0), fb = r * (j - J0);
  if (i < I1 && j >= jlo && j <= jhi) {
    const T t = cEx[j * cp + i] / (T)r;
    T* d = fEx + (size_t)fb * fp + fa;
    for (int q = 0; q < r; ++q) d[q] += t;
    cEx[j * cp + i] = T(0);
  }
  if (j < J1 && i >= ilo && i <= ihi) {
    const T t = cEy[j * cp + i] / (T)r;
    T* d = fEy + (size_t)fb * fp + fa;
    for (int q = 0; q < r; ++q) d[(size_t)q * fp] += t;
    cEy[j * cp + i] = T(0);
  }
}

// S2^T for one sample level: aE += 2 E_total aS2 (node weights), E0 share.
template <class T>
__global__ void ka_s2(T* aEx, T* aEy, const T* Ex, const T* Ey, const T* aS2, Step<T> c, int nx,
                      int ny, int p, double* e0acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double e0 = 0.0;
  if (i <= nx && j <= ny) {
    const int id = j * p + i;
    if (i < nx) {
      const T wl = (i > 0) ? T(0.5) : T(1);
      const T wr = (i + 1 < nx) ? T(0.5) : T(1);
      aEx[id] += T(2) * Ex[id] * (aS2[id] * wl + aS2[id + 1] * wr);
    }
    if (j < ny) {
      const T phi = c.sphi * c.ckx[i] - c.cphi * c.skx[i];
      const T ey = Ey[id] + c.E0 * phi;
      const T wb = (j > 0) ? T(0.5) : T(1);
      const T wt = (j + 1 < ny) ? T(0.5) : T(1);
      const T g = T(2) * ey * (aS2[id] * wb + aS2[id + p] * wt);
      aEy[id] += g;
      e0 += (double)g * (double)phi;
    }
  }
  const double s = block_sum_d(e0);
  if (threadIdx.x == 0 && threadIdx.y == 0 && s != 0.0) atomicAdd(e0acc, s);
}

// ---------------------------------------------------------------------------
// Continuity step (Eq. 4) reverse
// ---------------------------------------------------------------------------
// Per node: nu_net, D_eff and the derivatives the reverse sweep needs,
// evaluated exactly as k_rates does for the values.
template <class T>
__global__ void ka_rates_d(const T* n, const double* S2f, Dens d, double A1, int nx, int ny, int p, T* D,
                           T* nu, T* dDdn, T* dDdnu, T* dnudS2, T* nu_s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > nx || j > ny) return;
  const int id = j * p + i;
  const double s2 = S2f[id];
  const double e2 = eeff2_of(s2, d);
  const double eeff = sqrt(e2);
  const T x = ehp_of<T>(e2, d);
  T nui = T(0), dn = T(0), per_s = T(0);
  if (d.model == 1) {
    // Townsend form: nu = A p exp(-Bp/E) mu_e E, d nu/d S2 = nu (1 + Bp/E) / (2 S2)
    const T ee = sqrt((T)e2);
    if (ee > T(0)) {
      const T ex = exp(-(T)d.tBp / ee);
      nui = (T)d.A * ex * (T)d.mu_e * ee;
      per_s = (T)A1 * ex * (T)d.mu_e * ee;
      dn = (T)((double)nui * (1.0 + d.tBp / (double)ee) / (2.0 * s2));
    }
  } else if (x > T(0)) {
    const T ex = exp(T(-73.0) * pow(x, T(-0.44)));
    nui = (T)d.A * ex;
    per_s = (T)A1 * ex;
    // d nu / d S2 = nu 73 0.44 x^-1.44 (dx/dS2), dx/dS2 = 1 / (2 hp eeff N g)
    dn = (T)((double)nui * 73.0 * 0.44 * pow((double)x, -1.44) / (2.0 * d.hp * eeff * d.N * d.g));
  }
  const T nv = n[id];
  const T wp2 = nv * (T)d.wp2c;
  const T num = nui * (T)d.nu_m * (T)d.De + wp2 * (T)d.Da;
  const T den = nui * (T)d.nu_m + wp2;
  T Dv, gn = T(0), gnu = T(0);
  if (den == T(0)) {
    Dv = (T)d.De;
  } else {
    Dv = num / den;
    gn = (T)d.wp2c * ((T)d.Da - Dv) / den;
    gnu = (T)d.nu_m * ((T)d.De - Dv) / den;
  }
  D[id] = Dv;
  nu[id] = nui - (T)d.nu_a;
  dDdn[id] = gn;
  dDdnu[id] = gnu;
  dnudS2[id] = dn;
  nu_s[id] = per_s;
}

// Gather of a_n (old density), a_S2f and the s_nu share from a_n' (new
// density).  `dir` nodes of the fine mesh were set from the coarse mesh and do
// not depend on the fine density (their a_n' has been moved already).
template <class T>
__global__ void ka_density(const T* n, const T* D, const T* nu, const T* dDdn, const T* dDdnu,
                           const T* dnudS2, const T* nu_s, const T* an_new, T* an_old, T* aS2,
                           Dens d, Dir<T> dir, int nx, int ny, int p, double* snu_acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double sacc = 0.0;
  if (i <= nx && j <= ny) {
    const int id = j * p + i;
    auto isdir = [&](int a, int b) {
      return (dir.on[SIDE_BOTTOM] && b == 0) || (dir.on[SIDE_TOP] && b == ny) ||
             (dir.on[SIDE_LEFT] && a == 0) || (dir.on[SIDE_RIGHT] && a == nx);
    };
    const T T_ = (T)d.T, dx2 = (T)d.dx2, r = (T)d.r_ei;
    const T nk = n[id], Dk = D[id];
    T a_n = T(0), a_nu = T(0);
    const int nb_i[4] = {i + 1, i - 1, i, i};
    const int nb_j[4] = {j, j, j + 1, j - 1};
    const bool self_live = !isdir(i, j);
    const T ak = self_live ? an_new[id] : T(0);
    // own update
    if (self_live) {
      T dself = T(0), dnu = T(0);
      for (int f = 0; f < 4; ++f) {
        const int a = nb_i[f], b = nb_j[f];
        if (a < 0 || a > nx || b < 0 || b > ny) continue;
        const int fid = b * p + a;
        dself = dself + (T(0.5) * dDdn[id] * (n[fid] - nk) - T(0.5) * (Dk + D[fid]));
        dnu = dnu + T(0.5) * dDdnu[id] * (n[fid] - nk);
      }
      a_n = a_n + ak * (T(1) + T_ * (dself / dx2 + nu[id] - T(2) * r * nk));
      a_nu = a_nu + ak * T_ * (dnu / dx2 + nk);
    }
    // neighbours' updates that read this node
    for (int f = 0; f < 4; ++f) {
      const int a = nb_i[f], b = nb_j[f];
      if (a < 0 || a > nx || b < 0 || b > ny) continue;
      if (isdir(a, b)) continue;
      const int fid = b * p + a;
      const T af = an_new[fid];
      a_n = a_n + af * T_ * (T(0.5) * (D[fid] + Dk) + T(0.5) * dDdn[id] * (nk - n[fid])) / dx2;
      a_nu = a_nu + af * T_ * T(0.5) * dDdnu[id] * (nk - n[fid]) / dx2;
    }
    an_old[id] = a_n;
    aS2[id] = a_nu * dnudS2[id];
    sacc = (double)a_nu * (double)nu_s[id];
  }
  const double s = block_sum_d(sacc);
  if (threadIdx.x == 0 && threadIdx.y == 0 && s != 0.0) atomicAdd(snu_acc, s);
}

// a10^T: fine Dirichlet nodes took the new coarse density along the side
// (same side priority as k_density); their adjoint moves to the coarse mesh.
// Here dir.line[] point into the coarse adjoint array.
template <class T>
__global__ void ka_dir(T* an_f, int nfx, int nfy, int fp, Dir<T> dir) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > nfx || j > nfy) return;
  int sd = -1, q = 0;
  if (dir.on[SIDE_BOTTOM] && j == 0) { sd = SIDE_BOTTOM; q = i; }
  else if (dir.on[SIDE_TOP] && j == nfy) { sd = SIDE_TOP; q = i; }
  else if (dir.on[SIDE_LEFT] && i == 0) { sd = SIDE_LEFT; q = j; }
  else if (dir.on[SIDE_RIGHT] && i == nfx) { sd = SIDE_RIGHT; q = j; }
  if (sd < 0) return;
  const int id = j * fp + i;
  const T t = an_f[id];
  an_f[id] = T(0);
  double pos = (double)dir.start[sd] + (double)q / (double)dir.r;
  int i0 = (int)floor(pos);
  double w = pos - (double)i0;
  if (i0 < 0) { i0 = 0; w = 0.0; }
  if (i0 > dir.len[sd] - 2) { i0 = dir.len[sd] - 2; w = 1.0; }
  const T xp = (T)w;
  const int s = dir.stride[sd];
  T* l = const_cast<T*>(dir.line[sd]);
  atomicAdd(l + (size_t)i0 * s, t * (T(1) - xp));
  atomicAdd(l + (size_t)(i0 + 1) * s, t * xp);
}

// injection^T (commit^T): coarse nodes of the closed rectangle took the fine
// value; their adjoint goes to the coinciding fine node.
template <class T>
__global__ void ka_inject(T* an_c, int cp, T* an_f, int fp, int I0, int J0, int I1, int J1, int r) {
  const int i = I0 + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = J0 + blockIdx.y * blockDim.y + threadIdx.y;
  if (i > I1 || j > J1) return;
  const int cid = j * cp + i;
  an_f[(size_t)(r * (j - J0)) * fp + r * (i - I0)] += an_c[cid];
  an_c[cid] = T(0);
}

// a12^T: growth copied the old fine data and filled the rest bilinearly from
// the coarse mesh.  Adjoint: copy back to the old layout, scatter the rest.
template <class T>
struct ExpT {
  const T *nEx, *nEy, *nHz, *nvx, *nvy, *nn;   // adjoints in the new layout
  T *oEx, *oEy, *oHz, *ovx, *ovy, *on;         // adjoints in the old layout (written)
  T *cEx, *cEy, *cHz, *cvx, *cvy, *cn;         // coarse adjoints (atomic +=)
  int nnx, nny, np, onx, ony, op, cnx, cny, cp;
  int I0, J0, oI0, oJ0, r;
};

template <class T>
__device__ __forceinline__ void bilin_t(T* F, int p, int Lx, int Ly, double u, double v, T t) {
  int i0 = (int)floor(u);
  double fu = u - (double)i0;
  if (i0 < 0) { i0 = 0; fu = 0.0; }
  if (i0 > Lx - 2) { i0 = Lx - 2; fu = 1.0; }
  int j0 = (int)floor(v);
  double fv = v - (double)j0;
  if (j0 < 0) { j0 = 0; fv = 0.0; }
  if (j0 > Ly - 2) { j0 = Ly - 2; fv = 1.0; }
  T* r0 = F + (size_t)j0 * p;
  T* r1 = r0 + p;
  atomicAdd(r0 + i0, t * (T)((1.0 - fu) * (1.0 - fv)));
  atomicAdd(r0 + i0 + 1, t * (T)(fu * (1.0 - fv)));
  atomicAdd(r1 + i0, t * (T)((1.0 - fu) * fv));
  atomicAdd(r1 + i0 + 1, t * (T)(fu * fv));
}

template <class T>
__global__ void ka_expand(ExpT<T> e) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y * blockDim.y + threadIdx.y;
  if (a > e.nnx || b > e.nny) return;
  const int sa = a - e.r * (e.oI0 - e.I0), sb = b - e.r * (e.oJ0 - e.J0);
  const int id = b * e.np + a;
  const double rr = (double)e.r;
  const double xn = (double)e.I0 + (double)a / rr, yn = (double)e.J0 + (double)b / rr;
  const double xh = ((double)e.I0 + ((double)a + 0.5) / rr) - 0.5;
  const double yh = ((double)e.J0 + ((double)b + 0.5) / rr) - 0.5;
  const bool in_x = sa >= 0 && sa < e.onx, in_xn = sa >= 0 && sa <= e.onx;
  const bool in_y = sb >= 0 && sb < e.ony, in_yn = sb >= 0 && sb <= e.ony;
  const int oid = sb * e.op + sa;
  if (a < e.nnx) {
    if (in_x && in_yn) { e.oEx[oid] = e.nEx[id]; e.ovx[oid] = e.nvx[id]; }
    else {
      bilin_t(e.cEx, e.cp, e.cnx, e.cny + 1, xh, yn, e.nEx[id]);
      bilin_t(e.cvx, e.cp, e.cnx, e.cny + 1, xh, yn, e.nvx[id]);
    }
  }
  if (b < e.nny) {
    if (in_xn && in_y) { e.oEy[oid] = e.nEy[id]; e.ovy[oid] = e.nvy[id]; }
    else {
      bilin_t(e.cEy, e.cp, e.cnx + 1, e.cny, xn, yh, e.nEy[id]);
      bilin_t(e.cvy, e.cp, e.cnx + 1, e.cny, xn, yh, e.nvy[id]);
    }
  }
  if (a < e.nnx && b < e.nny) {
    if (in_x && in_y) e.oHz[oid] = e.nHz[id];
    else bilin_t(e.cHz, e.cp, e.cnx, e.cny, xh, yh, e.nHz[id]);
  }
  if (in_xn && in_yn) e.on[oid] = e.nn[id];
  else bilin_t(e.cn, e.cp, e.cnx + 1, e.cny + 1, xn, yn, e.nn[id]);
}

}  // namespace dmr
