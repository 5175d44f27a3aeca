// dmr_kernels.cuh -- sm_103a kernels of the DMR EM-plasma time step.
//
// Layout in HBM: every mesh array is row-major with y as the row index and a
// row pitch p (elements, a multiple of 64) shared by all arrays of the mesh:
//   Ex, vx [j*p + i], i < nx, j <= ny      Ey, vy [j*p + i], i <= nx, j < ny
//   Hz     [j*p + i], i < nx, j < ny       n, S2  [j*p + i], i <= nx, j <= ny
// Threads map x to threadIdx.x so each warp reads 32 consecutive elements.
//
// The stencils are HBM-bound (~0.7 flop/byte): no tensor cores.  Arithmetic
// is compiled without FMA contraction.  The update formulas of Eqs. 1-3 go
// through the helpers below, which every code path calls, so that the paths
// give identical bits: in FP32 they evaluate a * b + c with the product
// rounded first, in FP64 as one fused multiply-add (FP64 arithmetic, not
// HBM, bounds the FP64 launches on this part).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmr {

enum { SIDE_LEFT = 0, SIDE_RIGHT = 1, SIDE_BOTTOM = 2, SIDE_TOP = 3 };
enum { BC_MUR = 0, BC_CFB = 1, BC_PEC = 2 };

template <class T>
struct Mesh {
  T *Ex, *Ey, *Hz, *vx, *vy, *n;
  double* S2;
  int nx, ny;  // cells
  int p;       // row pitch (elements)
};

// Coefficients of one EM step on one mesh (Eqs. 1-3).
template <class T>
struct Step {
  T ch;        // dt / (mu0 dx)                 Faraday (Eq. 2)
  T ce;        // dt / (eps0 dx)                Ampere  (Eq. 1)
  T cj;        // dt e / (2 eps0): -J dt/eps0 = cj (n_a + n_b) v
  T va, vb;    // Crank-Nicolson momentum (Eq. 3): v' = va v - vb E
  T mur;       // (c dt - dx) / (c dt + dx)     first-order Mur
  T E0, sphi, cphi;      // incident amplitude and sin/cos of w t at this E level
  const T *ckx, *skx;    // cos(k x_i), sin(k x_i) of this mesh's node columns
  int accum;             // add |E_total|^2 of this level to S2
};

// Fine -> coarse transfer on the producer side (a8): the last fine sub-step
// of a coarse step, which computes the fine E^{n+1}, also writes the mean of
// each r collinear fine edges into the coarse E^{n+1} arrays (the coarse
// step's output, so the next coarse step reads plain arrays).  Ex: a shuffle
// over the r lanes of a column group; Ey: a running sum over r rows.  The
// sums are taken in the order q = 0 .. r-1, times 1/r.
template <class T>
struct RestrW {
  int on;
  T *cEx, *cEy;             // coarse E^{n+1}
  int cp;                   // coarse row pitch
  int I0, J0, I1, J1, r;
  int jlo, jhi, ilo, ihi;   // coarse Ex rows [jlo, jhi], Ey columns [ilo, ihi]
  T rinv;
  // coarse step of the persistent period: leave the edges that the last
  // fine sub-step writes (the box above) to it
  int skip;
};

// Coarse-fine boundary (Eq. 5b) for the fine mesh: per side, Mur or the
// coarse tangential-E line before (old) and after (new) the coarse step.
// With `recompute`, the new coarse values are evaluated from the coarse
// level-n state (cm, cc) with the coarse step's own arithmetic instead of
// being read, so a fine sub-step need not wait for the coarse step.
template <class T>
struct Bnd {
  int mode[4];              // BC_MUR, BC_CFB or BC_PEC (behind a CPML layer) per side
  const T* old_line[4];     // coarse tangential E at level n (strided)
  const T* new_line[4];     // coarse tangential E at level n+1 (strided)
  int stride[4];
  int len[4];               // coarse samples along the line
  int start[4];             // coarse index of the rectangle corner along the line
  int at[4];                // coarse row (bottom/top) or column (left/right) of the line
  int r;
  T frac;                   // k / r of the fine sub-step
  int recompute;
  Mesh<T> cm;
  Step<T> cc;
  // batched launches: sin/cos of the coarse phase per step of a period
  const T *cps, *cpc;
  int cN;
};

template <class T>
__device__ __forceinline__ T incident(const Step<T>& c, int i) {
  return c.E0 * (c.sphi * c.ckx[i] - c.cphi * c.skx[i]);
}

// a * b + c: FP32 with the product rounded first, FP64 fused
__device__ __forceinline__ float mad_(float a, float b, float c) { return a * b + c; }
__device__ __forceinline__ double mad_(double a, double b, double c) { return __fma_rn(a, b, c); }

// Eq. 2: Hz^{n+1/2} = Hz^{n-1/2} - ch curl, curl = dEy/dx - dEx/dy in cell units
template <class T>
__device__ __forceinline__ T upd_h(const Step<T>& c, T hzo, T curl) { return mad_(-c.ch, curl, hzo); }
// Eq. 3 (Crank-Nicolson momentum): v' = va v - vb E
template <class T>
__device__ __forceinline__ T upd_v(const Step<T>& c, T vo, T e) { return mad_(c.va, vo, -(c.vb * e)); }
// Eq. 1 at an x edge: Ex' = Ex + ce dH + cj (n_a + n_b) v'
template <class T>
__device__ __forceinline__ T upd_ex(const Step<T>& c, T exc, T dh, T ns, T v) {
  return mad_(c.cj * ns, v, mad_(c.ce, dh, exc));
}
// Eq. 1 at a y edge: Ey' = Ey - ce dH + cj (n_a + n_b) v'
template <class T>
__device__ __forceinline__ T upd_ey(const Step<T>& c, T eyc, T dh, T ns, T v) {
  return mad_(c.cj * ns, v, mad_(-c.ce, dh, eyc));
}
// mean of two squares, (a^2 + b^2) / 2
template <class T>
__device__ __forceinline__ T sq_mean(T a, T b) { return T(0.5) * mad_(a, a, b * b); }

// Squared total field at node (i, j): mean of the existing Ex^2 edges along x
// plus mean of the existing Ey^2 edges along y (incident added to Ey).
template <class T>
__device__ __forceinline__ T node_e2(const Mesh<T>& m, const Step<T>& c, int i, int j) {
  const int p = m.p;
  T sx, sy;
  if (i > 0 && i < m.nx) {
    T a = m.Ex[j * p + i - 1], b = m.Ex[j * p + i];
    sx = sq_mean(a, b);
  } else if (i > 0) {
    T a = m.Ex[j * p + i - 1];
    sx = a * a;
  } else {
    T b = m.Ex[j * p + i];
    sx = b * b;
  }
  T inc = incident(c, i);
  if (j > 0 && j < m.ny) {
    T e = m.Ey[(j - 1) * p + i] + inc, f = m.Ey[j * p + i] + inc;
    sy = sq_mean(e, f);
  } else if (j > 0) {
    T e = m.Ey[(j - 1) * p + i] + inc;
    sy = e * e;
  } else {
    T f = m.Ey[j * p + i] + inc;
    sy = f * f;
  }
  return sx + sy;
}

constexpr int TX = 32, TY = 8;   // 2-D thread block of the node-wise kernels

// Field loads of the EM step.  CG: through L2 only (ld.global.cg), for the
// persistent period kernel, whose blocks read what other blocks of the same
// launch wrote after a flag told them it is there; no L1 line or read-only
// cache path can then hold an older value.  Otherwise a plain load.
template <bool CG, class T>
__device__ __forceinline__ T ldv(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// E at an edge, 0 off the mesh
template <class T, bool CG = false>
__device__ __forceinline__ T load_ex(const Mesh<T>& m, int i, int j) {
  if (i < 0 || i >= m.nx || j < 0 || j > m.ny) return T(0);
  return ldv<CG>(m.Ex + j * m.p + i);
}

template <class T, bool CG = false>
__device__ __forceinline__ T load_ey(const Mesh<T>& m, int i, int j) {
  if (i < 0 || i > m.nx || j < 0 || j >= m.ny) return T(0);
  return ldv<CG>(m.Ey + j * m.p + i);
}

// Coarse E^{n+1} of interior coarse edge Ex(i, J) / Ey(I, j) evaluated from
// the level-n state with exactly the coarse step's operations (same values).
template <class T, bool CG = false>
__device__ __forceinline__ T coarse_new_ex(const Bnd<T>& b, int i, int J) {
  const Mesh<T>& m = b.cm;
  const Step<T>& c = b.cc;
  const int p = m.p;
  const T exm = load_ex<T, CG>(m, i, J - 1), exc = load_ex<T, CG>(m, i, J), exn = load_ex<T, CG>(m, i, J + 1);
  const T eym = load_ey<T, CG>(m, i, J - 1), eyc = load_ey<T, CG>(m, i, J);
  const T eymr = load_ey<T, CG>(m, i + 1, J - 1), eyr = load_ey<T, CG>(m, i + 1, J);
  const T hzp = upd_h(c, ldv<CG>(m.Hz + (J - 1) * p + i), (eymr - eym) - (exc - exm));
  const T hz = upd_h(c, ldv<CG>(m.Hz + J * p + i), (eyr - eyc) - (exn - exc));
  const T v = upd_v(c, ldv<CG>(m.vx + J * p + i), exc);
  return upd_ex(c, exc, hz - hzp, m.n[J * p + i] + m.n[J * p + i + 1], v);
}

template <class T, bool CG = false>
__device__ __forceinline__ T coarse_new_ey(const Bnd<T>& b, int I, int j) {
  const Mesh<T>& m = b.cm;
  const Step<T>& c = b.cc;
  const int p = m.p;
  const T eyl = load_ey<T, CG>(m, I - 1, j), eyc = load_ey<T, CG>(m, I, j), eyr = load_ey<T, CG>(m, I + 1, j);
  const T exl = load_ex<T, CG>(m, I - 1, j), exln = load_ex<T, CG>(m, I - 1, j + 1);
  const T exc = load_ex<T, CG>(m, I, j), exn = load_ex<T, CG>(m, I, j + 1);
  const T hzl = upd_h(c, ldv<CG>(m.Hz + j * p + I - 1), (eyc - eyl) - (exln - exl));
  const T hz = upd_h(c, ldv<CG>(m.Hz + j * p + I), (eyr - eyc) - (exn - exc));
  const T v = upd_v(c, ldv<CG>(m.vy + j * p + I), eyc + incident(c, I));
  return upd_ey(c, eyc, hz - hzl, m.n[j * p + I] + m.n[(j + 1) * p + I], v);
}

template <class T, bool CG = false>
__device__ __forceinline__ T coarse_new(const Bnd<T>& b, int sd, int k) {
  if (sd == SIDE_BOTTOM || sd == SIDE_TOP) return coarse_new_ex<T, CG>(b, k, b.at[sd]);
  return coarse_new_ey<T, CG>(b, b.at[sd], k);
}

// Eq. 5b for tangential sample q of side sd of the fine rectangle.  The
// fine sample sits at coarse position start + (q + 1/2)/r - 1/2 along the
// line = start + (2q + 1 - r)/(2r), split exactly into an index i0 and a
// weight xp (clamped to the line).
template <class T>
__device__ __forceinline__ int cfb_pos(const Bnd<T>& b, int sd, int q, T* xp_out) {
  const int num = 2 * q + 1 - b.r, den = 2 * b.r;
  const int fl = (num >= 0) ? num / den : -((-num + den - 1) / den);
  int i0 = b.start[sd] + fl;
  T xp = (T)(num - fl * den) / (T)den;
  if (i0 < 0) { i0 = 0; xp = T(0); }
  if (i0 > b.len[sd] - 2) { i0 = b.len[sd] - 2; xp = T(1); }
  *xp_out = xp;
  return i0;
}

// Eq. 5b: the coarse tangential E at level n (old line) interpolated in
// space at the sample, lo, blended in time with the level-n+1 one from n0, n1
// at coarse positions i0, i0 + 1.
template <class T, bool CG = false>
__device__ __forceinline__ T cfb_old(const Bnd<T>& b, int sd, int i0, T xp) {
  const T one = T(1);
  const T* o = b.old_line[sd];
  const int s = b.stride[sd];
  return ldv<CG>(o + i0 * s) * (one - xp) + ldv<CG>(o + (i0 + 1) * s) * xp;
}

template <class T>
__device__ __forceinline__ T cfb_blend(const Bnd<T>& b, T lo, T xp, T n0, T n1) {
  const T one = T(1);
  const T ln = n0 * (one - xp) + n1 * xp;
  return (one - b.frac) * lo + b.frac * ln;
}

// Programmatic dependent launch: an EM kernel lets the next EM launch of the
// stream be scheduled as soon as all its blocks have started, and waits for
// the previous one to complete (and its writes to be visible) before it
// touches memory.  Launched without the attribute both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// One EM step on one mesh, fused (a1-a6 + a5 of the level being left):
//   Hz^{n+1/2} from E^n (Eq. 2); S2 += |E^n_total|^2 at the nodes when c.accum;
//   v^{n+1/2} (Eq. 3); E^{n+1} on interior edges (Eq. 1); Mur on domain sides;
//   Eq. 5b on coarse-fine sides.
// E, H and v are double-buffered (read m.*, write d*), so strips may read
// neighbouring E^n, H^{n-1/2}, v^{n-1/2} while those are being advanced.
//
// Warp strips: lane L of a warp holds node column i = c0 - 1 + L with
// c0 = sw * strip (sw = STRIP_W, or the largest multiple of r up to it on the
// fine mesh); lanes 1..sw own their columns, lane 0 and lane sw + 1 are halo
// columns that only load and (lane 0) compute H for their neighbour.
// The warp marches up `rows` node rows, carrying the previous row's E^n, new
// H, density and Ey^n in registers; every x-neighbour comes by shuffle, so
// there is no shared memory and no block barrier (except in the last fine
// sub-step at one row per warp, whose warps sum the coarse Ey means in groups
// through shared memory).  A Mur side's boundary edge
// is advanced by the owner of the adjacent interior edge, which holds both E
// levels.  Each element is read once and written once: 60 B per cell (FP32).
constexpr int STRIP_W = 30;
constexpr int EM_WARPS = 4;   // warps per block (consecutive strips in y)
// resident EM blocks per SM the register allocation must allow: a 512^2
// coarse step with its fine sub-step is one wave of ~1200 blocks at 9 per SM
template <class T>
constexpr int kEmMinBlocks = sizeof(T) == 4 ? 9 : 6;

// CPML layer of the coarse mesh (Roden-Gedney recursion, kappa = 1): psi of
// the Hz curl terms along x and y at the cells, of the Ex (y) and Ey (x)
// curl terms at the edges, double-buffered like the fields (read level n,
// write level n+1); b, c per cell / node column and row (b = 1, c = 0
// outside the layer, where psi stays 0).
template <class T>
struct Pml {
  int on, L;
  const T *hx, *hy, *exy, *eyx;   // level n
  T *dhx, *dhy, *dexy, *deyx;      // level n+1
  const T *bxh, *cxh, *byh, *cyh, *bxn, *cxn, *byn, *cyn;
};

// Everything one EM step of one mesh needs; `gx` strips across x, `nblk`
// blocks (each EM_WARPS strips stacked in y).
template <class T>
struct EmArgs {
  Mesh<T> m;
  T *dEx, *dEy, *dHz, *dvx, *dvy;
  Step<T> c;
  Bnd<T> b;
  Pml<T> pml;
  RestrW<T> W;
  int sw;               // owned columns per strip (STRIP_W; a multiple of r on the fine mesh)
  int rows, gx, nblk;   // strips: rows per warp, strips across x, blocks
  int ncfb;             // blocks that write the coarse-fine boundary E (Eq. 5b)
  int lw;               // node columns per lane of the strips: 1 (em_strips) or 2 (em_strips2)
  // batched launches: the level-dependent fields (phase, E^2 sample, Eq. 5b
  // time weight) are filled in the kernel from the step index
  int kind;             // 0 coarse step, 1 fine sub-step
  int N, r;             // steps per period of this mesh, refinement factor
  const T *ps, *pc;     // sin / cos of w t for each step of a period
};

// Fill the level-dependent fields of a batched segment for coarse step m,
// sub-step k (1..r): the same values a single-run launch computes on the host.
template <class T>
__device__ __forceinline__ void em_set_level(EmArgs<T>& A, long long m, int k) {
  const long long level = A.kind == 0 ? m : (long long)A.r * m + (k - 1);
  const int q = (int)(level % A.N);
  A.c.sphi = A.ps[q];
  A.c.cphi = A.pc[q];
  A.c.accum = q != 0;
  if (A.kind == 1) {
    A.b.frac = (T)((double)k / (double)A.r);
    A.b.recompute = k == 1;
    const int qc = (int)(m % A.b.cN);
    A.b.cc.sphi = A.b.cps[qc];
    A.b.cc.cphi = A.b.cpc[qc];
    A.b.cc.accum = qc != 0;
  }
}

// Tangential E of the coarse-fine sides at the new level (a6, Eq. 5b).  It
// depends only on the coarse lines, not on this sub-step's interior update,
// so it runs as separate blocks of the same launch: one block per 32 *
// EM_WARPS consecutive samples of one side.  For the first sub-step of a
// coarse step (recompute) the coarse E^{n+1} at the positions the block's
// samples use is evaluated once per position into shared memory, then
// blended; later sub-steps read the stored level-n+1 line.
template <class T, bool CG = false>
__device__ __forceinline__ void em_cfb(const EmArgs<T>& A, int blk) {
  constexpr int NTH = 32 * EM_WARPS;
  __shared__ T cn[NTH + 2];
  const int nfx = A.m.nx, nfy = A.m.ny, p = A.m.p;
  const int order[4] = {SIDE_BOTTOM, SIDE_TOP, SIDE_LEFT, SIDE_RIGHT};
  int sd = -1, len = 0;
  for (int k = 0; k < 4; ++k) {
    if (A.b.mode[order[k]] != BC_CFB) continue;
    len = (order[k] == SIDE_BOTTOM || order[k] == SIDE_TOP) ? nfx : nfy;
    const int nb = (len + NTH - 1) / NTH;
    if (blk < nb) { sd = order[k]; break; }
    blk -= nb;
  }
  if (sd < 0) return;                          // whole block
  const int qa = blk * NTH, qb = min(qa + NTH, len) - 1;
  const int q = qa + (int)threadIdx.x;
  T xp = T(0);
  const int i0 = cfb_pos(A.b, sd, min(q, qb), &xp);
  const T lo = cfb_old<T, CG>(A.b, sd, i0, xp);        // in flight during the recompute
  T v;
  if (A.b.recompute) {
    T xa;
    const int c0 = cfb_pos(A.b, sd, qa, &xa), c1 = cfb_pos(A.b, sd, qb, &xa) + 1;
    for (int t = threadIdx.x; t <= c1 - c0; t += NTH) cn[t] = coarse_new<T, CG>(A.b, sd, c0 + t);
    __syncthreads();
    v = cfb_blend(A.b, lo, xp, cn[i0 - c0], cn[i0 + 1 - c0]);
  } else {
    const T* nl = A.b.new_line[sd];
    const int s = A.b.stride[sd];
    v = cfb_blend(A.b, lo, xp, ldv<CG>(nl + i0 * s), ldv<CG>(nl + (i0 + 1) * s));
  }
  if (q > qb) return;
  if (sd == SIDE_BOTTOM) A.dEx[q] = v;
  else if (sd == SIDE_TOP) A.dEx[nfy * p + q] = v;
  else if (sd == SIDE_LEFT) A.dEy[q * p] = v;
  else A.dEy[q * p + nfx] = v;
}

template <class T, bool PML, bool WR, bool CG, int RW = 0>
__device__ __forceinline__ void em_strips(const EmArgs<T>& A, int blk);

// Blocks of one mesh's EM step: the coarse-fine side blocks first (the
// longest dependent chain of the launch, so they are dispatched first), then
// the strips.
// PML: compile the CPML terms in (coarse launches of CPML runs only)
// WR: compile the producer-side fine->coarse transfer in (launches of the
// last fine sub-step of a coarse step only)
// CG: loads through L2 only (the persistent period kernel).  RW: the
// refinement factor of the fine->coarse transfer as a constant (0: read
// from the arguments), so its group sums unroll and its divisions are shifts.
template <class T, bool PML = false, bool WR = false, bool CG = false, int RW = 0>
__device__ __forceinline__ void em_segment(const EmArgs<T>& A, int blk) {
  if (blk < A.ncfb) em_cfb<T, CG>(A, blk);
  else em_strips<T, PML, WR, CG, RW>(A, blk - A.ncfb);
}

// em_strips for a block whose strips lie away from every side of the mesh:
// node columns c0 - 1 .. c0 + STRIP_W within [1, nx - 2] and node rows within
// [2, ny - 2] (so rows j0 - 1 .. j1 exist, no Mur, coarse-fine or PEC edge is
// near, every lane holds a column and every node's E^2 sample takes both
// neighbours).  The same operations as em_strips in the same order, without
// the edge tests.
template <class T>
__device__ __forceinline__ void em_strips_interior(const EmArgs<T>& A, int bx, int sy) {
  const Mesh<T>& m = A.m;
  T* __restrict__ dEx = A.dEx;
  T* __restrict__ dEy = A.dEy;
  T* __restrict__ dHz = A.dHz;
  T* __restrict__ dvx = A.dvx;
  T* __restrict__ dvy = A.dvy;
  const Step<T>& c = A.c;
  const int rows = A.rows;
  const int lane = threadIdx.x & 31;
  const int p = m.p;
  const int i = bx * STRIP_W - 1 + lane;
  const int j0 = sy * rows, j1 = j0 + rows;
  const bool own = lane >= 1 && lane <= STRIP_W;
  const T inc = incident(c, i);
  T exc = m.Ex[j0 * p + i], nc = m.n[j0 * p + i];
  T exp_, eyp, hzp;
  {
    const int q = (j0 - 1) * p + i;
    const T exm = m.Ex[q], eym = m.Ey[q], hzo = m.Hz[q];
    const T eyr = __shfl_down_sync(0xffffffffu, eym, 1);
    hzp = upd_h(c, hzo, (eyr - eym) - (exc - exm));
    exp_ = exm;
    eyp = eym;
  }
  struct Row { T exn, eyc, hzo, vxo, vyo, nn; double s2; };
  auto load_row = [&](int j) {
    Row q;
    const int id = j * p + i;
    q.exn = m.Ex[id + p];
    q.eyc = m.Ey[id];
    q.hzo = m.Hz[id];
    q.vxo = m.vx[id];
    q.vyo = m.vy[id];
    q.nn = m.n[id + p];
    q.s2 = (c.accum && own) ? m.S2[id] : 0.0;
    return q;
  };
  Row nxt = load_row(j0);
  for (int j = j0; j < j1; ++j) {
    const int id = j * p + i;
    const Row cur = nxt;
    if (j + 1 < j1) nxt = load_row(j + 1);
    const T exn = cur.exn, eyc = cur.eyc, hzo = cur.hzo, vxo = cur.vxo, vyo = cur.vyo, nn = cur.nn;
    const T eyr = __shfl_down_sync(0xffffffffu, eyc, 1);
    const T hz = upd_h(c, hzo, (eyr - eyc) - (exn - exc));
    const T hzl = __shfl_up_sync(0xffffffffu, hz, 1);
    const T exl = __shfl_up_sync(0xffffffffu, exc, 1);
    const T ncr = __shfl_down_sync(0xffffffffu, nc, 1);
    if (own) {
      dHz[id] = hz;
      if (c.accum) {
        const T sx = sq_mean(exl, exc);
        const T e = eyp + inc, f = eyc + inc;
        const T sy2 = sq_mean(e, f);
        m.S2[id] = cur.s2 + (double)(sx + sy2);
      }
      {
        const T v = upd_v(c, vxo, exc);
        dvx[id] = v;
        dEx[id] = upd_ex(c, exc, hz - hzp, nc + ncr, v);
      }
      {
        const T v = upd_v(c, vyo, eyc + inc);
        dvy[id] = v;
        dEy[id] = upd_ey(c, eyc, hz - hzl, nc + nn, v);
      }
    }
    exp_ = exc;
    exc = exn;
    eyp = eyc;
    hzp = hz;
    nc = nn;
  }
  (void)exp_;
}

template <class T, bool PML, bool WR, bool CG, int RW>
__device__ __forceinline__ void em_strips(const EmArgs<T>& A, int blk) {
  const Mesh<T>& m = A.m;
  T* __restrict__ dEx = A.dEx;
  T* __restrict__ dEy = A.dEy;
  T* __restrict__ dHz = A.dHz;
  T* __restrict__ dvx = A.dvx;
  T* __restrict__ dvy = A.dvy;
  const Step<T>& c = A.c;
  const Bnd<T>& b = A.b;
  const int rows = A.rows;
  const int lane = threadIdx.x & 31;
  const int bx = blk % A.gx, byb = blk / A.gx;
  const int sy = byb * EM_WARPS + (threadIdx.x >> 5);
  const int p = m.p, nx = m.nx, ny = m.ny;
  const int sw = A.sw;
  if constexpr (!PML && !WR && !CG) {
    // a block away from every side takes the path without edge tests
    const int bj0 = byb * EM_WARPS * rows, bj1 = bj0 + EM_WARPS * rows;
    if (sw == STRIP_W && bx * sw >= 2 && bx * sw + sw <= nx - 2 && bj0 >= 2 && bj1 <= ny - 1) {
      em_strips_interior<T>(A, bx, sy);
      return;
    }
  }
  const int i = bx * sw - 1 + lane;
  const int j0 = sy * rows;
  if (j0 > ny) return;                       // whole warp leaves together
  const int j1 = min(j0 + rows, ny + 1);     // node rows [j0, j1)
  const bool own = lane >= 1 && lane <= sw && i <= nx;
  // persistent period, coarse step: edges the last fine sub-step restricts
  // are left to it (only CG code reads the box)
  const RestrW<T>& Wk = A.W;
  auto keep_ex = [&](int ii, int jj) {
    return !(CG && Wk.skip && ii >= Wk.I0 && ii < Wk.I1 && jj >= Wk.jlo && jj <= Wk.jhi);
  };
  auto keep_ey = [&](int ii, int jj) {
    return !(CG && Wk.skip && ii >= Wk.ilo && ii <= Wk.ihi && jj >= Wk.J0 && jj < Wk.J1);
  };
  // CPML (warp-uniform): the strip's columns or rows reach into the layer
  const Pml<T>& P = A.pml;
  const int c0 = bx * sw;
  const bool pw = PML && P.on && (c0 - 1 <= P.L || c0 + sw >= nx - P.L || j0 - 1 <= P.L ||
                           j0 + rows >= ny - P.L);
  const bool live = lane <= sw + 1;          // lanes past the right halo idle
  const bool xcol = live && i >= 0 && i < nx;    // column has Ex / Hz
  const bool ycol = live && i >= 0 && i <= nx;   // column has Ey / n
  const T inc = ycol ? incident(c, i) : T(0);
  const T inc0 = incident(c, 0), incn = incident(c, nx);
  // ---- carried state for row j: Ex^n(j), Ex^n(j-1), Ey^n(j-1), Hz^{n+1/2}(j-1), n(j)
  T exc = T(0), exp_ = T(0), eyp = T(0), hzp = T(0), nc = T(0);
  if (xcol) exc = load_ex<T, CG>(m, i, j0);
  if (ycol) nc = m.n[j0 * p + i];
  if (j0 > 0) {
    // H of row j0-1, needed by the Ex update of row j0
    const int jm = j0 - 1;
    const T exm = xcol ? load_ex<T, CG>(m, i, jm) : T(0);
    const T eym = ycol ? load_ey<T, CG>(m, i, jm) : T(0);
    const T hzo = xcol ? ldv<CG>(m.Hz + jm * p + i) : T(0);
    const T eyr = __shfl_down_sync(0xffffffffu, eym, 1);
    if (xcol) {
      if (pw) {
        // the CPML-corrected H of row j0-1 (its owner stores psi)
        const int q = jm * p + i;
        const T dey = eyr - eym, dex = exc - exm;
        const T px = P.bxh[i] * ldv<CG>(P.hx + q) + P.cxh[i] * dey;
        const T py = P.byh[jm] * ldv<CG>(P.hy + q) + P.cyh[jm] * dex;
        hzp = upd_h(c, hzo, (dey + px) - (dex + py));
      } else {
        hzp = upd_h(c, hzo, (eyr - eym) - (exc - exm));
      }
    }
    exp_ = exm;
    eyp = eym;
  }
  // row loads, software-pipelined: row j+1 is loaded before row j is stored
  struct Row { T exn, eyc, hzo, vxo, vyo, nn; double s2; };
  auto load_row = [&](int j) {
    Row q;
    const int id = j * p + i;
    const bool in = j < ny;
    q.exn = (xcol && in) ? load_ex<T, CG>(m, i, j + 1) : T(0);
    q.eyc = (ycol && in) ? load_ey<T, CG>(m, i, j) : T(0);
    q.hzo = (xcol && in) ? ldv<CG>(m.Hz + id) : T(0);
    q.vxo = xcol ? ldv<CG>(m.vx + id) : T(0);
    q.vyo = (ycol && in) ? ldv<CG>(m.vy + id) : T(0);
    q.nn = (ycol && in) ? m.n[id + p] : T(0);
    q.s2 = (c.accum && own) ? ldv<CG>(m.S2 + id) : 0.0;
    return q;
  };
  Row nxt = load_row(j0);
  // a8 on the producer side: the column tests are fixed per lane; the row
  // phase jq = j mod r and the coarse row Jc = J0 + j / r are set once and
  // advance with j, so the loop divides by nothing.  An Ex group's r columns
  // are consecutive lanes of one strip (strip width a multiple of r).
  const int rw = WR ? (RW > 0 ? RW : A.W.r) : 1;
  const bool hx = WR && own && i < nx && (i % rw) == 0;                  // head of an Ex group
  const int Ic = WR ? A.W.I0 + (i > 0 ? i / rw : 0) : 0;
  const bool hy = hx && i > 0 && Ic >= A.W.ilo && Ic <= A.W.ihi;        // restricted Ey column
  // one row per warp (r dividing EM_WARPS): the r rows of a coarse row belong
  // to r consecutive warps of the block, which sum Ey through shared memory
  const bool cross = WR && rows == 1 && rw > 1;
  int jq = cross ? j0 % rw : 0, Jc = WR ? A.W.J0 + j0 / rw : 0;
  T eacc = T(0), eaccL = T(0), eaccR = T(0);   // Ey sums over the r rows of a coarse row
  for (int j = j0; j < j1; ++j) {
    const int id = j * p + i;
    const Row cur = nxt;
    if (j + 1 < j1) nxt = load_row(j + 1);
    const T exn = cur.exn, eyc = cur.eyc, hzo = cur.hzo, vxo = cur.vxo, vyo = cur.vyo, nn = cur.nn;
    const double s2 = cur.s2;
    // ---- H (Eq. 2)
    const T eyr = __shfl_down_sync(0xffffffffu, eyc, 1);
    T hz = T(0);
    if (xcol && j < ny) {
      if (pw) {
        const T dey = eyr - eyc, dex = exn - exc;
        const T px = P.bxh[i] * ldv<CG>(P.hx + id) + P.cxh[i] * dey;
        const T py = P.byh[j] * ldv<CG>(P.hy + id) + P.cyh[j] * dex;
        if (own) {
          P.dhx[id] = px;
          P.dhy[id] = py;
        }
        hz = upd_h(c, hzo, (dey + px) - (dex + py));
      } else {
        hz = upd_h(c, hzo, (eyr - eyc) - (exn - exc));
      }
    }
    const T hzl = __shfl_up_sync(0xffffffffu, hz, 1);
    const T exl = __shfl_up_sync(0xffffffffu, exc, 1);
    const T ncr = __shfl_down_sync(0xffffffffu, nc, 1);
    const T eyl = __shfl_up_sync(0xffffffffu, eyc, 1);
    const T vyl = __shfl_up_sync(0xffffffffu, vyo, 1);
    const T vyr = __shfl_down_sync(0xffffffffu, vyo, 1);
    T exw = T(0), exw0 = T(0), exwN = T(0), eyw = T(0), eywL = T(0), eywR = T(0);   // new E (a8)
    if (own) {
      if (i < nx && j < ny) dHz[id] = hz;
      // ---- S2 += |E^n|^2 at node (i, j)
      if (c.accum) {
        T sx, sy;
        if (i > 0 && i < nx) sx = sq_mean(exl, exc);
        else if (i > 0) sx = exl * exl;
        else sx = exc * exc;
        const T e = eyp + inc, f = eyc + inc;
        if (j > 0 && j < ny) sy = sq_mean(e, f);
        else if (j > 0) sy = e * e;
        else sy = f * f;
        m.S2[id] = s2 + (double)(sx + sy);
      }
      // ---- x edge (i, j)
      if (i < nx) {
        if (j > 0 && j < ny) {
          const T v = upd_v(c, vxo, exc);
          dvx[id] = v;
          T en;
          if (pw) {
            const T dh = hz - hzp;
            const T pe = P.byn[j] * ldv<CG>(P.exy + id) + P.cyn[j] * dh;
            P.dexy[id] = pe;
            en = upd_ex(c, exc, dh + pe, nc + ncr, v);
          } else {
            en = upd_ex(c, exc, hz - hzp, nc + ncr, v);
          }
          if (keep_ex(i, j)) dEx[id] = en;
          exw = en;
          if (j == 1 && b.mode[SIDE_BOTTOM] == BC_MUR) {
            dvx[i] = upd_v(c, ldv<CG>(m.vx + i), exp_);
            exw0 = exc + c.mur * (en - exp_);
            if (keep_ex(i, 0)) dEx[i] = exw0;
          }
          if (j == ny - 1 && b.mode[SIDE_TOP] == BC_MUR) {
            const int ib = ny * p + i;
            dvx[ib] = upd_v(c, ldv<CG>(m.vx + ib), exn);
            exwN = exc + c.mur * (en - exn);
            if (keep_ex(i, ny)) dEx[ib] = exwN;
          }
        } else {
          const int sd = (j == 0) ? SIDE_BOTTOM : SIDE_TOP;
          if (b.mode[sd] == BC_CFB) dvx[id] = upd_v(c, vxo, exc);  // E: em_cfb
          if (b.mode[sd] == BC_PEC) {
            dvx[id] = upd_v(c, vxo, exc);
            dEx[id] = T(0);
          }
        }
      }
      // ---- y edge (i, j)
      if (j < ny) {
        if (i > 0 && i < nx) {
          const T v = upd_v(c, vyo, eyc + inc);
          dvy[id] = v;
          T en;
          if (pw) {
            const T dh = hz - hzl;
            const T pe = P.bxn[i] * ldv<CG>(P.eyx + id) + P.cxn[i] * dh;
            P.deyx[id] = pe;
            en = upd_ey(c, eyc, dh + pe, nc + nn, v);
          } else {
            en = upd_ey(c, eyc, hz - hzl, nc + nn, v);
          }
          if (keep_ey(i, j)) dEy[id] = en;
          eyw = en;
          if (i == 1 && b.mode[SIDE_LEFT] == BC_MUR) {
            const int ib = j * p;
            dvy[ib] = upd_v(c, vyl, eyl + inc0);
            eywL = eyc + c.mur * (en - eyl);
            if (keep_ey(0, j)) dEy[ib] = eywL;
          }
          if (i == nx - 1 && b.mode[SIDE_RIGHT] == BC_MUR) {
            const int ib = j * p + nx;
            dvy[ib] = upd_v(c, vyr, eyr + incn);
            eywR = eyc + c.mur * (en - eyr);
            if (keep_ey(nx, j)) dEy[ib] = eywR;
          }
        } else {
          const int sd = (i == 0) ? SIDE_LEFT : SIDE_RIGHT;
          if (b.mode[sd] == BC_CFB) dvy[id] = upd_v(c, vyo, eyc + inc);  // E: em_cfb
          if (b.mode[sd] == BC_PEC) {
            dvy[id] = upd_v(c, vyo, eyc + inc);
            dEy[id] = T(0);
          }
        }
      }
    }
    if (WR && A.W.on) {
      // a8 on the producer side (last fine sub-step of a coarse step)
      const RestrW<T>& Wr = A.W;
      if (j > 0 && j < ny && jq == 0) {
        T acc = exw;
        for (int q = 1; q < rw; ++q) acc = acc + __shfl_down_sync(0xffffffffu, exw, q);
        if (hx && Jc >= Wr.jlo && Jc <= Wr.jhi) Wr.cEx[Jc * Wr.cp + Ic] = acc * Wr.rinv;
      }
      if (j == 1 && b.mode[SIDE_BOTTOM] == BC_MUR) {     // fine row 0 (Mur), coarse row J0
        T acc = exw0;
        for (int q = 1; q < rw; ++q) acc = acc + __shfl_down_sync(0xffffffffu, exw0, q);
        if (hx) Wr.cEx[Wr.J0 * Wr.cp + Ic] = acc * Wr.rinv;
      }
      if (j == ny - 1 && b.mode[SIDE_TOP] == BC_MUR) {   // fine row ny (Mur), coarse row J1
        T acc = exwN;
        for (int q = 1; q < rw; ++q) acc = acc + __shfl_down_sync(0xffffffffu, exwN, q);
        if (hx) Wr.cEx[Wr.J1 * Wr.cp + Ic] = acc * Wr.rinv;
      }
      if (j < ny && cross) {
        // the group's rows are all below ny (ny and the group start are
        // multiples of r), so all r warps of the group arrive here; named
        // barrier 1 + group index (barrier 0 is __syncthreads'), 32 r threads
        __shared__ T sey[EM_WARPS][32], slr[EM_WARPS][2];
        const int wq = threadIdx.x >> 5, w0 = wq - jq;
        sey[wq][lane] = eyw;
        if (own && i == 1) slr[wq][0] = eywL;
        if (own && i == nx - 1) slr[wq][1] = eywR;
        // immediate barrier ids: the block then reserves barriers 0..2 only,
        // not all sixteen, which would cap the blocks resident on an SM
        static_assert(EM_WARPS == 4, "r = 2: two groups of two warps; r = 4: one group of four");
        if (rw == 4) asm volatile("bar.sync 1, 128;" ::: "memory");
        else if (w0 == 0) asm volatile("bar.sync 1, 64;" ::: "memory");
        else asm volatile("bar.sync 2, 64;" ::: "memory");
        if (jq == rw - 1) {
          eacc = sey[w0][lane];
          for (int q = 1; q < rw; ++q) eacc = eacc + sey[w0 + q][lane];
          if (hy) Wr.cEy[Jc * Wr.cp + Ic] = eacc * Wr.rinv;
          if (own && i == 1 && b.mode[SIDE_LEFT] == BC_MUR) {
            eaccL = slr[w0][0];
            for (int q = 1; q < rw; ++q) eaccL = eaccL + slr[w0 + q][0];
            Wr.cEy[Jc * Wr.cp + Wr.I0] = eaccL * Wr.rinv;
          }
          if (own && i == nx - 1 && b.mode[SIDE_RIGHT] == BC_MUR) {
            eaccR = slr[w0][1];
            for (int q = 1; q < rw; ++q) eaccR = eaccR + slr[w0 + q][1];
            Wr.cEy[Jc * Wr.cp + Wr.I1] = eaccR * Wr.rinv;
          }
        }
      } else if (j < ny) {
        eacc = jq == 0 ? eyw : eacc + eyw;
        eaccL = jq == 0 ? eywL : eaccL + eywL;
        eaccR = jq == 0 ? eywR : eaccR + eywR;
        if (jq == rw - 1) {
          if (hy) Wr.cEy[Jc * Wr.cp + Ic] = eacc * Wr.rinv;
          if (own && i == 1 && b.mode[SIDE_LEFT] == BC_MUR) Wr.cEy[Jc * Wr.cp + Wr.I0] = eaccL * Wr.rinv;
          if (own && i == nx - 1 && b.mode[SIDE_RIGHT] == BC_MUR) Wr.cEy[Jc * Wr.cp + Wr.I1] = eaccR * Wr.rinv;
        }
      }
      if (++jq == rw) { jq = 0; ++Jc; }
    }
    exp_ = exc;
    exc = exn;
    eyp = eyc;
    hzp = hz;
    nc = nn;
  }
}

// ---- two node columns per lane (FP32) ---------------------------------------
// The same EM step as em_strips (Eqs. 1-3, Mur, the E^2 sample of the level
// being left, the producer-side a8 transfer) with each lane holding two
// adjacent node columns, so each row's loads and stores are 8-byte vector
// accesses (16-byte for the FP64 E^2 sums) and one lane shuffle serves two
// nodes: a warp covers 64 columns, lanes 1..STRIP_W2/2 own 60 of them, lane 0
// and lane 31 hold the halo columns.  Every element is computed by the same
// operations in the same order as em_strips, so results are the same bits.
// Used for Mur/coarse-fine/PEC sides without CPML, outside the persistent
// period; the last fine sub-step (WR) takes r = 2 or 4 with rows per warp a
// multiple of r.  The v of every edge is stored by the owner of its column
// and row (on a Mur side that is the value em_strips' neighbour stores).
constexpr int STRIP_W2 = 60;

__device__ __forceinline__ float2 ld_f2(const float* q, bool both, bool first) {
  float2 v = make_float2(0.f, 0.f);
  if (both) v = *reinterpret_cast<const float2*>(q);
  else if (first) v.x = *q;
  return v;
}
__device__ __forceinline__ double2 ld_d2(const double* q, bool both, bool first) {
  double2 v = make_double2(0.0, 0.0);
  if (both) v = *reinterpret_cast<const double2*>(q);
  else if (first) v.x = *q;
  return v;
}
__device__ __forceinline__ void st_f2(float* q, float a, float b, bool sa, bool sb) {
  if (sa && sb) {
    *reinterpret_cast<float2*>(q) = make_float2(a, b);
  } else {
    if (sa) q[0] = a;
    if (sb) q[1] = b;
  }
}
__device__ __forceinline__ void st_d2(double* q, double a, double b, bool sa, bool sb) {
  if (sa && sb) {
    *reinterpret_cast<double2*>(q) = make_double2(a, b);
  } else {
    if (sa) q[0] = a;
    if (sb) q[1] = b;
  }
}

// |E^n|^2 at node (i, j) from the x edges left/right and the y edges
// below/above (incident added), as em_strips takes it
__device__ __forceinline__ float node_e2_sample(int i, int j, int nx, int ny, float exl, float exc,
                                                float eyp, float eyc, float inc) {
  float sx, sy;
  if (i > 0 && i < nx) sx = sq_mean(exl, exc);
  else if (i > 0) sx = exl * exl;
  else sx = exc * exc;
  const float e = eyp + inc, f = eyc + inc;
  if (j > 0 && j < ny) sy = sq_mean(e, f);
  else if (j > 0) sy = e * e;
  else sy = f * f;
  return sx + sy;
}

// One node column of a row of em_strips2: the x and y edge updates of node
// (i, j) from its loaded and neighbouring values (the operations of em_strips)
struct Col2 {
  float en_x, en_y;   // E^{n+1} of the node's x / y edge (interior edges)
  float exw0, exwN;   // Mur bottom / top: the boundary row's new Ex
  float eywL, eywR;   // Mur left / right: the boundary column's new Ey
};

__device__ __forceinline__ Col2 col2_update(const Step<float>& c, const Bnd<float>& b, int i, int j,
                                            int nx, int ny, float hz, float hzp, float hzl,
                                            float exc, float exp_, float exn, float eyc, float eyl,
                                            float eyr, float vxo, float vyo, float nc, float ncr,
                                            float nn, float inc) {
  Col2 o;
  o.en_x = o.en_y = o.exw0 = o.exwN = o.eywL = o.eywR = 0.f;
  if (i < nx && j > 0 && j < ny) {
    const float v = upd_v(c, vxo, exc);
    const float en = upd_ex(c, exc, hz - hzp, nc + ncr, v);
    o.en_x = en;
    if (j == 1 && b.mode[SIDE_BOTTOM] == BC_MUR) o.exw0 = exc + c.mur * (en - exp_);
    if (j == ny - 1 && b.mode[SIDE_TOP] == BC_MUR) o.exwN = exc + c.mur * (en - exn);
  }
  if (j < ny && i > 0 && i < nx) {
    const float v = upd_v(c, vyo, eyc + inc);
    const float en = upd_ey(c, eyc, hz - hzl, nc + nn, v);
    o.en_y = en;
    if (i == 1 && b.mode[SIDE_LEFT] == BC_MUR) o.eywL = eyc + c.mur * (en - eyl);
    if (i == nx - 1 && b.mode[SIDE_RIGHT] == BC_MUR) o.eywR = eyc + c.mur * (en - eyr);
  }
  return o;
}

// em_strips2 for a block away from every side of the mesh: node columns
// c0 - 2 .. c0 + 61 within [1, nx - 2] and node rows within [2, ny - 2], so
// every lane holds two valid columns and no Mur, coarse-fine or PEC edge is
// near.  The same operations in the same order, without the edge tests.
template <bool WR, int RW>
__device__ __forceinline__ void em_strips2_interior(const EmArgs<float>& A, int bx, int sy) {
  const Mesh<float>& m = A.m;
  float* __restrict__ dEx = A.dEx;
  float* __restrict__ dEy = A.dEy;
  float* __restrict__ dHz = A.dHz;
  float* __restrict__ dvx = A.dvx;
  float* __restrict__ dvy = A.dvy;
  const Step<float>& c = A.c;
  const int rows = A.rows;
  const int lane = threadIdx.x & 31;
  const int p = m.p;
  const int ia = bx * STRIP_W2 - 2 + 2 * lane;
  const int j0 = sy * rows, j1 = j0 + rows;
  const bool lo = lane >= 1 && lane <= STRIP_W2 / 2;
  const float inc_a = incident(c, ia), inc_b = incident(c, ia + 1);
  float2 exc = *reinterpret_cast<const float2*>(m.Ex + j0 * p + ia);
  float2 nc = *reinterpret_cast<const float2*>(m.n + j0 * p + ia);
  float2 eyp, hzp;
  {
    const int q = (j0 - 1) * p + ia;
    const float2 exm = *reinterpret_cast<const float2*>(m.Ex + q);
    const float2 eym = *reinterpret_cast<const float2*>(m.Ey + q);
    const float2 hzo = *reinterpret_cast<const float2*>(m.Hz + q);
    const float eyr_b = __shfl_down_sync(0xffffffffu, eym.x, 1);
    hzp.x = upd_h(c, hzo.x, (eym.y - eym.x) - (exc.x - exm.x));
    hzp.y = upd_h(c, hzo.y, (eyr_b - eym.y) - (exc.y - exm.y));
    eyp = eym;
  }
  struct Row2 { float2 exn, eyc, hzo, vxo, vyo, nn; double2 s2; };
  auto load_row = [&](int j) {
    Row2 q;
    const int id = j * p + ia;
    q.exn = *reinterpret_cast<const float2*>(m.Ex + id + p);
    q.eyc = *reinterpret_cast<const float2*>(m.Ey + id);
    q.hzo = *reinterpret_cast<const float2*>(m.Hz + id);
    q.vxo = *reinterpret_cast<const float2*>(m.vx + id);
    q.vyo = *reinterpret_cast<const float2*>(m.vy + id);
    q.nn = *reinterpret_cast<const float2*>(m.n + id + p);
    q.s2 = (c.accum && lo) ? *reinterpret_cast<const double2*>(m.S2 + id) : make_double2(0.0, 0.0);
    return q;
  };
  Row2 nxt = load_row(j0);
  constexpr int rw = WR ? RW : 1;
  const bool hx = WR && lo && (ia % rw) == 0;
  const int Ic = WR ? A.W.I0 + ia / rw : 0;
  const bool hy = hx && Ic >= A.W.ilo && Ic <= A.W.ihi;
  int jq = 0, Jc = WR ? A.W.J0 + j0 / rw : 0;
  float eacc_a = 0.f;
  for (int j = j0; j < j1; ++j) {
    const int id = j * p + ia;
    const Row2 cur = nxt;
    if (j + 1 < j1) nxt = load_row(j + 1);
    const float eyr_b = __shfl_down_sync(0xffffffffu, cur.eyc.x, 1);
    float2 hz;
    hz.x = upd_h(c, cur.hzo.x, (cur.eyc.y - cur.eyc.x) - (cur.exn.x - exc.x));
    hz.y = upd_h(c, cur.hzo.y, (eyr_b - cur.eyc.y) - (cur.exn.y - exc.y));
    const float hzl_a = __shfl_up_sync(0xffffffffu, hz.y, 1);
    const float exl_a = __shfl_up_sync(0xffffffffu, exc.y, 1);
    const float ncr_b = __shfl_down_sync(0xffffffffu, nc.x, 1);
    const float vxa = upd_v(c, cur.vxo.x, exc.x), vxb = upd_v(c, cur.vxo.y, exc.y);
    const float enxa = upd_ex(c, exc.x, hz.x - hzp.x, nc.x + nc.y, vxa);
    const float enxb = upd_ex(c, exc.y, hz.y - hzp.y, nc.y + ncr_b, vxb);
    const float vya = upd_v(c, cur.vyo.x, cur.eyc.x + inc_a);
    const float vyb = upd_v(c, cur.vyo.y, cur.eyc.y + inc_b);
    const float enya = upd_ey(c, cur.eyc.x, hz.x - hzl_a, nc.x + cur.nn.x, vya);
    const float enyb = upd_ey(c, cur.eyc.y, hz.y - hz.x, nc.y + cur.nn.y, vyb);
    if (lo) {
      *reinterpret_cast<float2*>(dHz + id) = hz;
      if (c.accum) {
        float sx = sq_mean(exl_a, exc.x);
        float e = eyp.x + inc_a, f = cur.eyc.x + inc_a;
        const float e2a = sx + sq_mean(e, f);
        sx = sq_mean(exc.x, exc.y);
        e = eyp.y + inc_b;
        f = cur.eyc.y + inc_b;
        const float e2b = sx + sq_mean(e, f);
        *reinterpret_cast<double2*>(m.S2 + id) = make_double2(cur.s2.x + (double)e2a, cur.s2.y + (double)e2b);
      }
      *reinterpret_cast<float2*>(dvx + id) = make_float2(vxa, vxb);
      *reinterpret_cast<float2*>(dEx + id) = make_float2(enxa, enxb);
      *reinterpret_cast<float2*>(dvy + id) = make_float2(vya, vyb);
      *reinterpret_cast<float2*>(dEy + id) = make_float2(enya, enyb);
    }
    if (WR && A.W.on) {
      const RestrW<float>& Wr = A.W;
      if (jq == 0) {
        float acc = enxa + enxb;
        if (rw == 4) {
          acc = acc + __shfl_down_sync(0xffffffffu, enxa, 1);
          acc = acc + __shfl_down_sync(0xffffffffu, enxb, 1);
        }
        if (hx && Jc >= Wr.jlo && Jc <= Wr.jhi) Wr.cEx[Jc * Wr.cp + Ic] = acc * Wr.rinv;
      }
      eacc_a = jq == 0 ? enya : eacc_a + enya;
      if (jq == rw - 1 && hy) Wr.cEy[Jc * Wr.cp + Ic] = eacc_a * Wr.rinv;
      if (++jq == rw) { jq = 0; ++Jc; }
    }
    exc = cur.exn;
    eyp = cur.eyc;
    hzp = hz;
    nc = cur.nn;
  }
}

template <bool WR, int RW>
__device__ __forceinline__ void em_strips2(const EmArgs<float>& A, int blk) {
  const Mesh<float>& m = A.m;
  float* __restrict__ dEx = A.dEx;
  float* __restrict__ dEy = A.dEy;
  float* __restrict__ dHz = A.dHz;
  float* __restrict__ dvx = A.dvx;
  float* __restrict__ dvy = A.dvy;
  const Step<float>& c = A.c;
  const Bnd<float>& b = A.b;
  const int rows = A.rows;
  const int lane = threadIdx.x & 31;
  const int bx = blk % A.gx, byb = blk / A.gx;
  const int sy = byb * EM_WARPS + (threadIdx.x >> 5);
  const int p = m.p, nx = m.nx, ny = m.ny;
  const int sw = A.sw;                       // owned columns per strip (even)
  {
    // a block away from every side takes the path without edge tests
    const int bj0 = byb * EM_WARPS * rows, bj1 = bj0 + EM_WARPS * rows;
    if (sw == STRIP_W2 && bx * sw >= 3 && bx * sw + 63 <= nx && bj0 >= 2 && bj1 <= ny - 1) {
      em_strips2_interior<WR, RW>(A, bx, sy);
      return;
    }
  }
  const int ia = bx * sw - 2 + 2 * lane, ib = ia + 1;
  const int j0 = sy * rows;
  if (j0 > ny) return;                       // whole warp leaves together
  const int j1 = min(j0 + rows, ny + 1);
  const bool lo = lane >= 1 && 2 * lane <= sw;
  const bool own_a = lo && ia <= nx, own_b = lo && ib <= nx;
  const bool live = 2 * lane <= sw + 2;
  const bool xa = live && ia >= 0 && ia < nx, xb = live && ib >= 0 && ib < nx;
  const bool ya = live && ia >= 0 && ia <= nx, yb = live && ib >= 0 && ib <= nx;
  const float inc_a = ya ? incident(c, ia) : 0.f, inc_b = yb ? incident(c, ib) : 0.f;
  const bool pec_b = b.mode[SIDE_BOTTOM] == BC_PEC, pec_t = b.mode[SIDE_TOP] == BC_PEC;
  const bool pec_l = b.mode[SIDE_LEFT] == BC_PEC, pec_r = b.mode[SIDE_RIGHT] == BC_PEC;
  // carried state for row j: Ex^n(j), Ex^n(j-1), Ey^n(j-1), Hz^{n+1/2}(j-1), n(j)
  float2 exc = ld_f2(m.Ex + j0 * p + ia, xb, xa);
  float2 nc = ld_f2(m.n + j0 * p + ia, yb, ya);
  float2 exp_ = make_float2(0.f, 0.f), eyp = make_float2(0.f, 0.f), hzp = make_float2(0.f, 0.f);
  if (j0 > 0) {
    const int jm = j0 - 1;
    const float2 exm = ld_f2(m.Ex + jm * p + ia, xb, xa);
    const float2 eym = ld_f2(m.Ey + jm * p + ia, yb, ya);
    const float2 hzo = ld_f2(m.Hz + jm * p + ia, xb, xa);
    const float eyr_b = __shfl_down_sync(0xffffffffu, eym.x, 1);
    if (xa) hzp.x = upd_h(c, hzo.x, (eym.y - eym.x) - (exc.x - exm.x));
    if (xb) hzp.y = upd_h(c, hzo.y, (eyr_b - eym.y) - (exc.y - exm.y));
    exp_ = exm;
    eyp = eym;
  }
  struct Row2 { float2 exn, eyc, hzo, vxo, vyo, nn; double2 s2; };
  auto load_row = [&](int j) {
    Row2 q;
    const int id = j * p + ia;
    const bool in = j < ny;
    const float2 z = make_float2(0.f, 0.f);
    q.exn = in ? ld_f2(m.Ex + id + p, xb, xa) : z;
    q.eyc = in ? ld_f2(m.Ey + id, yb, ya) : z;
    q.hzo = in ? ld_f2(m.Hz + id, xb, xa) : z;
    q.vxo = ld_f2(m.vx + id, xb, xa);
    q.vyo = in ? ld_f2(m.vy + id, yb, ya) : z;
    q.nn = in ? ld_f2(m.n + id + p, yb, ya) : z;
    q.s2 = c.accum ? ld_d2(m.S2 + id, own_b, own_a) : make_double2(0.0, 0.0);
    return q;
  };
  Row2 nxt = load_row(j0);
  // a8 on the producer side (r = 2 or 4, rows a multiple of r): an Ex group
  // of r columns is one lane (r = 2) or two (r = 4, heads on odd lanes)
  constexpr int rw = WR ? RW : 1;
  static_assert(!WR || RW == 2 || RW == 4, "two columns per lane: r = 2 or 4");
  const bool hx = WR && own_a && ia < nx && (ia % rw) == 0;         // head of an Ex group
  const int Ic = WR ? A.W.I0 + (ia > 0 ? ia / rw : 0) : 0;
  const bool hy = hx && ia > 0 && Ic >= A.W.ilo && Ic <= A.W.ihi;   // restricted Ey column
  int jq = 0, Jc = WR ? A.W.J0 + j0 / rw : 0;
  float eacc_a = 0.f, eaccL = 0.f, eaccR = 0.f;
  for (int j = j0; j < j1; ++j) {
    const int id = j * p + ia;
    const Row2 cur = nxt;
    if (j + 1 < j1) nxt = load_row(j + 1);
    // ---- H (Eq. 2)
    const float eyr_b = __shfl_down_sync(0xffffffffu, cur.eyc.x, 1);
    float2 hz = make_float2(0.f, 0.f);
    if (j < ny) {
      if (xa) hz.x = upd_h(c, cur.hzo.x, (cur.eyc.y - cur.eyc.x) - (cur.exn.x - exc.x));
      if (xb) hz.y = upd_h(c, cur.hzo.y, (eyr_b - cur.eyc.y) - (cur.exn.y - exc.y));
    }
    const float hzl_a = __shfl_up_sync(0xffffffffu, hz.y, 1);
    const float exl_a = __shfl_up_sync(0xffffffffu, exc.y, 1);
    const float ncr_b = __shfl_down_sync(0xffffffffu, nc.x, 1);
    const float vyr_b = __shfl_down_sync(0xffffffffu, cur.vyo.x, 1);
    const Col2 oa = col2_update(c, b, ia, j, nx, ny, hz.x, hzp.x, hzl_a, exc.x, exp_.x, cur.exn.x,
                                cur.eyc.x, 0.f, cur.eyc.y, cur.vxo.x, cur.vyo.x, nc.x, nc.y,
                                cur.nn.x, inc_a);
    const Col2 ob = col2_update(c, b, ib, j, nx, ny, hz.y, hzp.y, hz.x, exc.y, exp_.y, cur.exn.y,
                                cur.eyc.y, cur.eyc.x, eyr_b, cur.vxo.y, cur.vyo.y, nc.y, ncr_b,
                                cur.nn.y, inc_b);
    const bool ax = own_a && ia < nx, bxx = own_b && ib < nx;   // columns with an x edge
    // ---- stores: H, the E^2 sample of level n, v, interior and PEC E
    st_f2(dHz + id, hz.x, hz.y, ax && j < ny, bxx && j < ny);
    if (c.accum) {
      const float e2a = node_e2_sample(ia, j, nx, ny, exl_a, exc.x, eyp.x, cur.eyc.x, inc_a);
      const float e2b = node_e2_sample(ib, j, nx, ny, exc.x, exc.y, eyp.y, cur.eyc.y, inc_b);
      st_d2(m.S2 + id, cur.s2.x + (double)e2a, cur.s2.y + (double)e2b, own_a, own_b);
    }
    st_f2(dvx + id, upd_v(c, cur.vxo.x, exc.x), upd_v(c, cur.vxo.y, exc.y), ax, bxx);
    {
      const bool xin = j > 0 && j < ny;
      const bool xpec = (j == 0 && pec_b) || (j == ny && pec_t);
      st_f2(dEx + id, oa.en_x, ob.en_x, ax && (xin || xpec), bxx && (xin || xpec));
      if (j == 1 && b.mode[SIDE_BOTTOM] == BC_MUR) st_f2(dEx + ia, oa.exw0, ob.exw0, ax && j < ny, bxx && j < ny);
      if (j == ny - 1 && b.mode[SIDE_TOP] == BC_MUR) st_f2(dEx + ny * p + ia, oa.exwN, ob.exwN, ax && j > 0, bxx && j > 0);
    }
    if (j < ny) {
      st_f2(dvy + id, upd_v(c, cur.vyo.x, cur.eyc.x + inc_a), upd_v(c, cur.vyo.y, cur.eyc.y + inc_b),
            own_a, own_b);
      const bool ia_in = ia > 0 && ia < nx, ib_in = ib > 0 && ib < nx;
      const bool ia_pec = (ia == 0 && pec_l) || (ia == nx && pec_r);
      const bool ib_pec = (ib == 0 && pec_l) || (ib == nx && pec_r);
      st_f2(dEy + id, oa.en_y, ob.en_y, own_a && (ia_in || ia_pec), own_b && (ib_in || ib_pec));
      // Mur left / right: the boundary column's Ey by the owner of column 1 / nx - 1
      if (own_b && ib == 1 && b.mode[SIDE_LEFT] == BC_MUR) dEy[j * p] = ob.eywL;
      if (own_a && ia == nx - 1 && b.mode[SIDE_RIGHT] == BC_MUR) dEy[j * p + nx] = oa.eywR;
      if (own_b && ib == nx - 1 && b.mode[SIDE_RIGHT] == BC_MUR) dEy[j * p + nx] = ob.eywR;
    }
    if (WR && A.W.on) {
      // a8 on the producer side, sums in the order of em_strips
      const RestrW<float>& Wr = A.W;
      auto gsum = [&](float va_, float vb_) {
        float acc = va_ + vb_;
        if (rw == 4) {
          acc = acc + __shfl_down_sync(0xffffffffu, va_, 1);
          acc = acc + __shfl_down_sync(0xffffffffu, vb_, 1);
        }
        return acc;
      };
      if (j > 0 && j < ny && jq == 0) {
        const float acc = gsum(oa.en_x, ob.en_x);
        if (hx && Jc >= Wr.jlo && Jc <= Wr.jhi) Wr.cEx[Jc * Wr.cp + Ic] = acc * Wr.rinv;
      }
      if (j == 1 && b.mode[SIDE_BOTTOM] == BC_MUR) {     // fine row 0 (Mur), coarse row J0
        const float acc = gsum(oa.exw0, ob.exw0);
        if (hx) Wr.cEx[Wr.J0 * Wr.cp + Ic] = acc * Wr.rinv;
      }
      if (j == ny - 1 && b.mode[SIDE_TOP] == BC_MUR) {   // fine row ny (Mur), coarse row J1
        const float acc = gsum(oa.exwN, ob.exwN);
        if (hx) Wr.cEx[Wr.J1 * Wr.cp + Ic] = acc * Wr.rinv;
      }
      if (j < ny) {
        const float eR = ia == nx - 1 ? oa.eywR : ob.eywR;
        eacc_a = jq == 0 ? oa.en_y : eacc_a + oa.en_y;
        eaccL = jq == 0 ? ob.eywL : eaccL + ob.eywL;
        eaccR = jq == 0 ? eR : eaccR + eR;
        if (jq == rw - 1) {
          if (hy) Wr.cEy[Jc * Wr.cp + Ic] = eacc_a * Wr.rinv;
          if (own_b && ib == 1 && b.mode[SIDE_LEFT] == BC_MUR) Wr.cEy[Jc * Wr.cp + Wr.I0] = eaccL * Wr.rinv;
          if (((own_a && ia == nx - 1) || (own_b && ib == nx - 1)) && b.mode[SIDE_RIGHT] == BC_MUR)
            Wr.cEy[Jc * Wr.cp + Wr.I1] = eaccR * Wr.rinv;
        }
      }
      if (++jq == rw) { jq = 0; ++Jc; }
    }
    exp_ = exc;
    exc = cur.exn;
    eyp = cur.eyc;
    hzp = hz;
    nc = cur.nn;
  }
}

// resident blocks per SM the two-column kernels' registers allow
constexpr int kEm2MinBlocks = 6;

template <bool WR = false, int RW = 0>
__device__ __forceinline__ void em_segment2(const EmArgs<float>& A, int blk) {
  if (blk < A.ncfb) em_cfb<float>(A, blk);
  else em_strips2<WR, RW>(A, blk - A.ncfb);
}

// k_em with two node columns per lane (FP32, no CPML)
template <bool WR = false, int RW = 0>
__global__ void __launch_bounds__(32 * EM_WARPS, kEm2MinBlocks) k_em_w2(EmArgs<float> A) {
  pdl_enter();
  em_segment2<WR, RW>(A, blockIdx.x);
}


template <class T, bool PML = false, bool WR = false, int RW = 0>
__global__ void __launch_bounds__(32 * EM_WARPS, kEmMinBlocks<T>) k_em(EmArgs<T> A) {
  pdl_enter();
  em_segment<T, PML, WR, false, RW>(A, blockIdx.x);
}

constexpr int kSegStage = 256;   // segment offsets staged in shared memory up to this many

// Batched EM launch: segment s (one mesh of one run) owns blocks
// [off[s], off[s+1]); its arguments come from a table in device memory.
template <class T, bool WR = false>
__global__ void __launch_bounds__(32 * EM_WARPS, 5) k_em_batch(const EmArgs<T>* __restrict__ tab,
                                                            const int* __restrict__ off, int nseg,
                                                            long long m, int k) {
  __shared__ EmArgs<T> A;
  __shared__ int seg, base;
  __shared__ int soff[kSegStage + 1];
  const int b = (int)blockIdx.x;
  if (nseg <= kSegStage) {
    // one coalesced load of the offsets, then a parallel scan: the segment
    // q with off[q] <= b < off[q+1] (empty segments never match)
    for (int q = threadIdx.x; q <= nseg; q += blockDim.x) soff[q] = off[q];
    __syncthreads();
    for (int q = threadIdx.x; q < nseg; q += blockDim.x)
      if (soff[q] <= b && b < soff[q + 1]) { seg = q; base = soff[q]; }
  } else if (threadIdx.x == 0) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    seg = lo;
    base = off[lo];
  }
  __syncthreads();
  {
    const int* src = reinterpret_cast<const int*>(tab + seg);
    int* dst = reinterpret_cast<int*>(&A);
    for (int q = threadIdx.x; q < (int)(sizeof(EmArgs<T>) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) em_set_level(A, m, k);
  __syncthreads();
  em_segment<T, false, WR>(A, b - base);
}

// Two independent EM steps in one launch: the coarse step A0 and the first
// fine sub-step A1, whose coarse boundary values are recomputed.  The fine
// blocks come first in the grid (their side blocks carry the launch's
// longest dependent chain).
template <class T, bool PML = false>
__global__ void __launch_bounds__(32 * EM_WARPS, kEmMinBlocks<T>) k_em2(EmArgs<T> A0, EmArgs<T> A1) {
  pdl_enter();
  const int n1 = A1.nblk + A1.ncfb;   // the fine sub-step's blocks first
  if ((int)blockIdx.x < n1) em_segment(A1, blockIdx.x);
  else em_segment<T, PML>(A0, blockIdx.x - n1);
}

// ----------------------------------------------------------------------------
// Period end: E_eff, rates, continuity step, totals, flags (a9-a11, a13)
// ----------------------------------------------------------------------------
struct Dens {
  double N;          // EM samples per period on this mesh
  double g;          // 1 + (w/nu_m)^2
  double hp;         // 100 p: E_eff/p in V/(cm Torr)
  double A;          // s_nu 5.14e11 p (air fit) or s_nu A_T p (Townsend form)
  double nu_m, nu_a, De, Da;
  double wp2c;       // e^2/(m eps0)
  double heat;       // e^2/(m nu_m): period-mean J.E = n heat E_eff^2
  double T;          // period
  double dx2;        // dx^2
  double r_ei;
  double invN, invg, inv_hp;   // 1/N, 1/g, 1/hp
  int model;                   // 0 air fit, 1 Townsend form
  double tBp, mu_e;            // Townsend: B p (V/m), mobility e/(m_e nu_m)
};

// E_eff^2 of a node from its FP64 running E^2 sum of the period:
// E_rms^2 = S2 / N, E_eff^2 = E_rms^2 / (1 + (w/nu_m)^2) (Sec. II.B).  FP64
// multiplies by host reciprocals: divides and square roots in FP64 are slow
// software sequences on this GPU.
__device__ __forceinline__ double eeff2_of(double s2, const Dens& d) { return s2 * d.invN * d.invg; }

// E_eff / p in V/(cm Torr), the argument of the ionization fit, in the run's
// precision
template <class T>
__device__ __forceinline__ T ehp_of(double e2, const Dens& d) { return sqrt((T)e2) * (T)d.inv_hp; }

// Ionization frequency nu_i at E_eff^2 = e2 (Sec. II.A), in the run's
// precision: the air fit of E_eff/p, or the Townsend form
// s_nu A p exp(-B p / E_eff) mu_e E_eff; 0 where E_eff = 0
template <class T>
__device__ __forceinline__ T nu_ion(double e2, const Dens& d) {
  if (d.model == 1) {
    const T ee = sqrt((T)e2);
    return ee > T(0) ? (T)d.A * exp(-(T)d.tBp / ee) * (T)d.mu_e * ee : T(0);
  }
  const T x = ehp_of<T>(e2, d);
  return (x > T(0)) ? (T)d.A * exp(T(-73.0) * pow(x, T(-0.44))) : T(0);
}

// composite trapezoid weight of node (i, j): coarse mesh outside the
// rectangle, fine mesh inside it
struct Wts {
  int nx, ny;               // cells of this mesh
  int has_rect;             // coarse mesh with a fine rectangle
  int I0, J0, I1, J1;
};

__device__ __forceinline__ double trap_w(const Wts& w, int i, int j) {
  double wx = (i == 0 || i == w.nx) ? 0.5 : 1.0;
  double wy = (j == 0 || j == w.ny) ? 0.5 : 1.0;
  double v = wx * wy;
  if (w.has_rect) {
    double px = (i < w.I0 || i > w.I1) ? 0.0 : ((i == w.I0 || i == w.I1) ? 0.5 : 1.0);
    double py = (j < w.J0 || j > w.J1) ? 0.0 : ((j == w.J0 || j == w.J1) ? 0.5 : 1.0);
    v = v - px * py;
  }
  return v;
}

// deterministic block sum of a double (blockDim.x*blockDim.y threads, <= 1024)
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int nt = blockDim.x * blockDim.y;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((t & 31) == 0) sh[t >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (t < 32) {
    s = (t < (nt + 31) / 32) ? sh[t] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;  // valid in thread 0
}

struct Ctl {           // device control block
  double st[8];        // 0 N_e, 1 P_abs, 2 W_abs, 3 periods, 4 n_max
  int bbox[4];         // imin, jmin, imax, jmax of the flags
  int nflag;
  int err;
  int side;            // threshold-line hits: bit 0 left, 1 bottom, 2 right, 3 top
  unsigned done;       // blocks of the period's last launch that have written their partials
};

// One mesh's part of the period-end launches: its blocks are 2-D tiles of
// TX x TY nodes, gx tiles across, nb in all.
template <class T>
struct PeMesh {
  Mesh<T> m;
  Step<T> c;           // level of the period's last E^2 sample
  Dens d;
  Wts w;
  T *D, *nu, *ntmp, *erms;
  double *partP, *partN;
  int gx, nb;
};

// Dirichlet (coarse-fine) sides of the fine density step: new coarse density
// interpolated along the side (Eq. 5b, frac = 1).
template <class T>
struct Dir {
  int on[4];            // side is a coarse-fine boundary
  const T* line[4];     // new coarse density along the side (strided; adjoint)
  int stride[4];
  int len[4];
  int start[4];
  int at[4];            // coarse row (bottom/top) or column (left/right) of the side
  int r;
};

// The arguments of the three period-end launches.
template <class T>
struct PeArgs {
  PeMesh<T> C, F;       // coarse mesh; fine rectangle (F.nb = 0 when there is none)
  Dir<T> dir;           // the fine density's coarse-fine sides
  int r;
  int4 rect;            // the rectangle's corner nodes (coarse)
  T n_th, gs;           // flags: threshold density, 1/(2 dx g_th)
  uint8_t* mask;
  Ctl* ctl;
  double dxc2, dxf2, period;   // cell areas, EM period
  unsigned* sched;             // the persistent period's counters and flags, cleared here
  int nsched;
};

// node (i, j) of mesh-block b of a PeMesh (false past the mesh)
template <class T>
__device__ __forceinline__ bool pe_node(const PeMesh<T>& M, int b, int* i, int* j) {
  const int by = b / M.gx, bx = b - by * M.gx;
  *i = bx * TX + (int)threadIdx.x;
  *j = by * TY + (int)threadIdx.y;
  return *i <= M.m.nx && *j <= M.m.ny;
}

// a9 first pass at node (i, j): finish the period's S2 with the last level,
// E_eff, nu_net, D_eff; E_rms of the period kept in erms (E_rms^2 = S2 / N,
// the output E_rms(x, y, t)); reset S2.  Returns the node's period-mean
// absorbed-power term.
template <class T>
__device__ __forceinline__ double rates_node(const PeMesh<T>& M, int i, int j) {
  const Mesh<T>& m = M.m;
  const Dens& d = M.d;
  const int id = j * m.p + i;
  const double s2 = m.S2[id] + (double)node_e2(m, M.c, i, j);
  const double e2 = eeff2_of(s2, d);
  const T nui = nu_ion<T>(e2, d);
  T n = m.n[id];
  T wp2 = n * (T)d.wp2c;
  T num = nui * (T)d.nu_m * (T)d.De + wp2 * (T)d.Da;
  T den = nui * (T)d.nu_m + wp2;
  M.D[id] = (den == T(0)) ? (T)d.De : num / den;
  M.nu[id] = nui - (T)d.nu_a;
  M.erms[id] = sqrt((T)(s2 * d.invN));
  m.S2[id] = 0.0;
  return trap_w(M.w, i, j) * (double)n * d.heat * e2;
}

// a9 second pass at node (i, j): forward-Euler continuity step over one
// period with face-mean D_eff, zero flux through the domain edges.
template <class T>
__device__ __forceinline__ T density_new(const PeMesh<T>& M, int i, int j) {
  const Mesh<T>& m = M.m;
  const int p = m.p;
  const int id = j * p + i;
  const T* D = M.D;
  const T n = m.n[id];
  const T Di = D[id];
  T lap = T(0);
  if (i < m.nx) lap = lap + T(0.5) * (Di + D[id + 1]) * (m.n[id + 1] - n);
  if (i > 0) lap = lap + T(0.5) * (Di + D[id - 1]) * (m.n[id - 1] - n);
  if (j < m.ny) lap = lap + T(0.5) * (Di + D[id + p]) * (m.n[id + p] - n);
  if (j > 0) lap = lap + T(0.5) * (Di + D[id - p]) * (m.n[id - p] - n);
  const T rate = lap / (T)M.d.dx2 + M.nu[id] * n - (T)M.d.r_ei * n * n;
  return n + (T)M.d.T * rate;
}

// a10: fine node q of side sd from the new coarse density at the two coarse
// nodes of the side's line around it (Eq. 5b, frac = 1), the coarse values
// evaluated here with the coarse step's own operations
template <class T>
__device__ __forceinline__ T dir_value(const Dir<T>& d, const PeMesh<T>& C, int sd, int q) {
  double pos = (double)d.start[sd] + (double)q / (double)d.r;
  int i0 = (int)floor(pos);
  double w = pos - (double)i0;
  if (i0 < 0) { i0 = 0; w = 0.0; }
  if (i0 > d.len[sd] - 2) { i0 = d.len[sd] - 2; w = 1.0; }
  const T xp = (T)w;
  const bool hor = sd == SIDE_BOTTOM || sd == SIDE_TOP;
  const T a = hor ? density_new(C, i0, d.at[sd]) : density_new(C, d.at[sd], i0);
  const T b = hor ? density_new(C, i0 + 1, d.at[sd]) : density_new(C, d.at[sd], i0 + 1);
  return a * (T(1) - xp) + b * xp;
}

// Period end, launch 1 (a9 first pass, a13 power): the coarse mesh's blocks,
// then the fine rectangle's; resets the control block.
template <class T>
__global__ void __launch_bounds__(TX * TY) k_pe_rates(PeArgs<T> A) {
  const int b = (int)blockIdx.x;
  if (b == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    Ctl* ctl = A.ctl;
    ctl->bbox[0] = 0x7fffffff; ctl->bbox[1] = 0x7fffffff;
    ctl->bbox[2] = -1; ctl->bbox[3] = -1;
    ctl->nflag = 0; ctl->st[4] = 0.0; ctl->side = 0; ctl->done = 0u;
  }
  // the persistent period launch that may follow starts from zero counts
  for (int k = b * (TX * TY) + threadIdx.y * TX + threadIdx.x; k < A.nsched; k += gridDim.x * TX * TY)
    A.sched[k] = 0u;
  const bool fine = b >= A.C.nb;
  const PeMesh<T>& M = fine ? A.F : A.C;
  const int mb = fine ? b - A.C.nb : b;
  int i, j;
  double contrib = 0.0;
  if (pe_node(M, mb, &i, &j)) contrib = rates_node(M, i, j);
  const double s = block_sum(contrib);
  if (threadIdx.x == 0 && threadIdx.y == 0) M.partP[mb] = s;
}

// Period end, launch 2 (a9 second pass, a10): the new density of both meshes;
// the fine nodes of coarse-fine sides take the interpolated new coarse density.
template <class T>
__global__ void __launch_bounds__(TX * TY) k_pe_density(PeArgs<T> A) {
  const int b = (int)blockIdx.x;
  const bool fine = b >= A.C.nb;
  const PeMesh<T>& M = fine ? A.F : A.C;
  int i, j;
  if (!pe_node(M, fine ? b - A.C.nb : b, &i, &j)) return;
  const int id = j * M.m.p + i;
  if (fine) {
    const Dir<T>& d = A.dir;
    if (d.on[SIDE_BOTTOM] && j == 0) { M.ntmp[id] = dir_value(d, A.C, SIDE_BOTTOM, i); return; }
    if (d.on[SIDE_TOP] && j == M.m.ny) { M.ntmp[id] = dir_value(d, A.C, SIDE_TOP, i); return; }
    if (d.on[SIDE_LEFT] && i == 0) { M.ntmp[id] = dir_value(d, A.C, SIDE_LEFT, j); return; }
    if (d.on[SIDE_RIGHT] && i == M.m.nx) { M.ntmp[id] = dir_value(d, A.C, SIDE_RIGHT, j); return; }
  }
  M.ntmp[id] = density_new(M, i, j);
}

// the new coarse density at node (i, j) as the commit writes it: the fine
// value at nodes of the closed rectangle (direct copy, Sec. III.C)
template <class T>
__device__ __forceinline__ T committed_coarse(const PeArgs<T>& A, int i, int j) {
  const int4 rc = A.rect;
  if (A.F.nb > 0 && i >= rc.x && i <= rc.z && j >= rc.y && j <= rc.w)
    return A.F.ntmp[(size_t)(A.r * (j - rc.y)) * A.F.m.p + A.r * (i - rc.x)];
  return A.C.ntmp[j * A.C.m.p + i];
}

// a11 at coarse node (i, j) of the committed density: flag (threshold OR
// central gradient, the latter as (dn_x s)^2 + (dn_y s)^2 > 1 with
// s = 1/(2 dx g_th)), mask, bounding box, count, largest density,
// threshold-line hits of the rectangle's sides (Sec. III.D)
template <class T>
__device__ __forceinline__ void flag_node(const PeArgs<T>& A, int i, int j, T n) {
  const Mesh<T>& m = A.C.m;
  Ctl* ctl = A.ctl;
  bool f = n > A.n_th;
  if (i > 0 && i < m.nx && j > 0 && j < m.ny) {
    T gx = (committed_coarse(A, i + 1, j) - committed_coarse(A, i - 1, j)) * A.gs;
    T gy = (committed_coarse(A, i, j + 1) - committed_coarse(A, i, j - 1)) * A.gs;
    f = f || (gx * gx + gy * gy > T(1));
  }
  A.mask[(size_t)j * (m.nx + 1) + i] = f ? 1 : 0;
  // largest density (non-negative doubles order like their bit patterns)
  const double dn = (double)n;
  if (dn != dn) {
    atomicOr(&ctl->err, 1);
  } else if (dn > 0.0) {
    atomicMax((unsigned long long*)&ctl->st[4], (unsigned long long)__double_as_longlong(dn));
  }
  const int4 rc = A.rect;
  if (n > A.n_th) {
    const bool in_y = j >= rc.y && j <= rc.w, in_x = i >= rc.x && i <= rc.z;
    const int bits = (i == rc.x && in_y ? 1 : 0) | (j == rc.y && in_x ? 2 : 0) |
                     (i == rc.z && in_y ? 4 : 0) | (j == rc.w && in_x ? 8 : 0);
    if (bits) atomicOr(&ctl->side, bits);
  }
  if (f) {
    atomicMin(&ctl->bbox[0], i);
    atomicMin(&ctl->bbox[1], j);
    atomicMax(&ctl->bbox[2], i);
    atomicMax(&ctl->bbox[3], j);
    atomicAdd(&ctl->nflag, 1);
  }
}

// deterministic sum of v[0..n) by one block (thread 0 gets the result)
__device__ __forceinline__ double block_sum_array(const double* v, int n) {
  double a = 0.0;
  const int t = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  for (int q = t; q < n; q += nt) a += v[q];
  return block_sum(a);
}

// Period end, launch 3 (commit, a11, a13 totals): both meshes take their new
// density, the coarse nodes of the closed rectangle the fine one; electron
// partials; flags on the coarse mesh (a fine rectangle only); the last block
// to finish sums all partials in a fixed order into the FP64 totals.
template <class T>
__global__ void __launch_bounds__(TX * TY) k_pe_commit(PeArgs<T> A) {
  __shared__ bool last;
  const int b = (int)blockIdx.x;
  const bool fine = b >= A.C.nb;
  const PeMesh<T>& M = fine ? A.F : A.C;
  const int mb = fine ? b - A.C.nb : b;
  int i, j;
  double contrib = 0.0;
  if (pe_node(M, mb, &i, &j)) {
    const T v = fine ? M.ntmp[j * M.m.p + i] : committed_coarse(A, i, j);
    M.m.n[j * M.m.p + i] = v;
    contrib = trap_w(M.w, i, j) * (double)v;
    if (!fine && A.F.nb > 0) flag_node(A, i, j, v);
  }
  const double s = block_sum(contrib);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    M.partN[mb] = s;
    __threadfence();
    last = atomicAdd(&A.ctl->done, 1u) == (unsigned)(A.C.nb + A.F.nb) - 1u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const double sPc = block_sum_array(A.C.partP, A.C.nb);
  const double sPf = block_sum_array(A.F.partP, A.F.nb);
  const double sNc = block_sum_array(A.C.partN, A.C.nb);
  const double sNf = block_sum_array(A.F.partN, A.F.nb);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    Ctl* ctl = A.ctl;
    const double P = A.dxc2 * sPc + A.dxf2 * sPf;
    const double N = A.dxc2 * sNc + A.dxf2 * sNf;
    ctl->st[0] = N;
    ctl->st[1] = P;
    ctl->st[2] = ctl->st[2] + P * A.period;
    ctl->st[3] = ctl->st[3] + 1.0;
    if (!(N == N) || !(P == P)) ctl->err |= 1;
    ctl->done = 0u;
  }
}

// ----------------------------------------------------------------------------
// Growth (a12) and set-up
// ----------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T bilin(const T* F, int p, int Lx, int Ly, double u, double v) {
  int i0 = (int)floor(u);
  double fu = u - (double)i0;
  if (i0 < 0) { i0 = 0; fu = 0.0; }
  if (i0 > Lx - 2) { i0 = Lx - 2; fu = 1.0; }
  int j0 = (int)floor(v);
  double fv = v - (double)j0;
  if (j0 < 0) { j0 = 0; fv = 0.0; }
  if (j0 > Ly - 2) { j0 = Ly - 2; fv = 1.0; }
  const T a = (T)((1.0 - fu) * (1.0 - fv)), b = (T)(fu * (1.0 - fv));
  const T cc = (T)((1.0 - fu) * fv), dd = (T)(fu * fv);
  const T* r0 = F + (size_t)j0 * p;
  const T* r1 = r0 + p;
  return r0[i0] * a + r0[i0 + 1] * b + r1[i0] * cc + r1[i0 + 1] * dd;
}

// New fine arrays of rectangle (I0, J0) with (nf.nx, nf.ny) cells: values of
// the old rectangle are copied, the rest bilinear from coarse (Eq. 5a).
// The E_rms of the last period (nerms, oerms, cerms on the new fine, old fine
// and coarse node grids) is filled the same way as the density.
template <class T>
__global__ void k_expand(Mesh<T> nf, Mesh<T> of, Mesh<T> c, int I0, int J0, int oI0, int oJ0,
                         int has_old, int r, T* nerms, const T* oerms, const T* cerms) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y * blockDim.y + threadIdx.y;
  if (a > nf.nx || b > nf.ny) return;
  const int sa = a - r * (oI0 - I0), sb = b - r * (oJ0 - J0);
  const int id = b * nf.p + a;
  const double rr = (double)r;
  const double xn = (double)I0 + (double)a / rr, yn = (double)J0 + (double)b / rr;
  const double xh = ((double)I0 + ((double)a + 0.5) / rr) - 0.5;
  const double yh = ((double)J0 + ((double)b + 0.5) / rr) - 0.5;
  const bool in_x = has_old && sa >= 0 && sa < of.nx;
  const bool in_xn = has_old && sa >= 0 && sa <= of.nx;
  const bool in_y = has_old && sb >= 0 && sb < of.ny;
  const bool in_yn = has_old && sb >= 0 && sb <= of.ny;
  const int oid = sb * of.p + sa;
  if (a < nf.nx) {  // Ex, vx at (i+1/2, j)
    if (in_x && in_yn) {
      nf.Ex[id] = of.Ex[oid];
      nf.vx[id] = of.vx[oid];
    } else {
      nf.Ex[id] = bilin(c.Ex, c.p, c.nx, c.ny + 1, xh, yn);
      nf.vx[id] = bilin(c.vx, c.p, c.nx, c.ny + 1, xh, yn);
    }
  }
  if (b < nf.ny) {  // Ey, vy at (i, j+1/2)
    if (in_xn && in_y) {
      nf.Ey[id] = of.Ey[oid];
      nf.vy[id] = of.vy[oid];
    } else {
      nf.Ey[id] = bilin(c.Ey, c.p, c.nx + 1, c.ny, xn, yh);
      nf.vy[id] = bilin(c.vy, c.p, c.nx + 1, c.ny, xn, yh);
    }
  }
  if (a < nf.nx && b < nf.ny) {
    nf.Hz[id] = (in_x && in_y) ? of.Hz[oid] : bilin(c.Hz, c.p, c.nx, c.ny, xh, yh);
  }
  nf.n[id] = (in_xn && in_yn) ? of.n[oid] : bilin(c.n, c.p, c.nx + 1, c.ny + 1, xn, yn);
  nerms[id] = (in_xn && in_yn) ? oerms[oid] : bilin(cerms, c.p, c.nx + 1, c.ny + 1, xn, yn);
  nf.S2[id] = 0.0;
}

template <class T>
__global__ void k_seed(Mesh<T> m, int gi0, int gj0, double dx, double n0, double x0, double y0,
                       double sx, double sy, int add) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > m.nx || j > m.ny) return;
  const double x = (double)(gi0 + i) * dx, y = (double)(gj0 + j) * dx;
  const double ux = x - x0, uy = y - y0;
  const double arg = ux * ux / (sx * sx) + uy * uy / (sy * sy);
  const double g = (arg <= 60.0) ? n0 * exp(-fmin(arg, 60.0)) : 0.0;
  const int id = j * m.p + i;
  m.n[id] = add ? (T)((double)m.n[id] + g) : (T)g;
}

// direct copy of the fine density into the coinciding coarse nodes
template <class T>
__global__ void k_inject(Mesh<T> c, Mesh<T> f, int I0, int J0, int I1, int J1, int r) {
  const int i = I0 + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = J0 + blockIdx.y * blockDim.y + threadIdx.y;
  if (i > I1 || j > J1) return;
  c.n[j * c.p + i] = f.n[(size_t)(r * (j - J0)) * f.p + r * (i - I0)];
}

// running S2 through the present E level (S2 holds the levels before it)
template <class T>
__global__ void k_s2_view(Mesh<T> m, Step<T> c, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > m.nx || j > m.ny) return;
  out[j * m.p + i] = m.S2[j * m.p + i] + (double)node_e2(m, c, i, j);
}

// E_rms within a period: the RMS over the q samples of the running sum, the
// present E level added on the fly (out in the run's precision, same pitch)
template <class T>
__global__ void k_erms_view(Mesh<T> m, Step<T> c, double q, T* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > m.nx || j > m.ny) return;
  const double s2 = m.S2[j * m.p + i] + (double)node_e2(m, c, i, j);
  out[j * m.p + i] = (T)sqrt(s2 / q);
}

// strided 2-D copy between a dense buffer and a pitched array (device side)
template <class E>
__global__ void k_copy2d(E* dst, int dp, const E* src, int sp, int cols, int rows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= cols || j >= rows) return;
  dst[(size_t)j * dp + i] = src[(size_t)j * sp + i];
}

}  // namespace dmr
