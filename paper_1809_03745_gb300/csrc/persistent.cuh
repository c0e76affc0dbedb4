// persistent.cuh -- the whole solve in one cooperative launch.
//
// Multigrid phases (arXiv:1809.03745, Sec. 3.3.2) run as grid-stride loops
// separated by a software grid barrier; levels small enough for one CTA run
// inside CTA 0 with block barriers while the other CTAs wait; the coarsest
// level is solved by a precomputed dense inverse.  The FP64 outer loop
// (residual, convergence test ||r||_inf <= tol ||b||_inf of Sec. 3.3.2,
// update) runs on the device, so a solve needs no host round trip.
#pragma once

#include "mg_kernels.cuh"

namespace ebp {

constexpr int MAXLEV = 16;
constexpr int PT = 512;                          // threads per CTA of the persistent kernel
constexpr long long BAR_WAIT_CYCLES = 4000000000LL;  // ~2 s of SM clock: a barrier wait gives up after this

// Tile-streamed passes over large 3D levels (sweep3d.cuh): tiles of SW_TX x
// SW_TY cells, boxes with a halo of SW_HX cells in x (16 bytes of 4-byte
// data, the TMA alignment of the x coordinate) and SW_HY in y, flag boxes
// SW_FBX bytes wide from SW_FHX cells left of the tile (16-byte alignment of
// bytes); two planes per copy, a ring of SW_NS two-plane slots.
constexpr int SW_TX = 32, SW_TY = 32, SW_HX = 4, SW_BX = SW_TX + 2 * SW_HX, SW_HY = 2, SW_FHX = 16, SW_FBX = 64;
constexpr int SW_NS = 6;  // three slots in use, three copies in flight
// shared-memory head before the ring: SW_NS mbarriers, a failure flag, and
// from SW_QOFF a queue of SW_QN item indices (the order the items arrive in)
constexpr int SW_QOFF = 64, SW_QN = 8, SW_HEAD = 128;
static_assert(8 * SW_NS + 4 <= SW_QOFF && SW_QOFF + 4 * SW_QN <= SW_HEAD, "sweep head layout");

template <class T>
struct SweepLev {
  int on;       // 1: the level relaxes by tile-streamed sweeps, x -> alt
  int rs;       // 1: and restricts by the tile-streamed residual + restriction
  int zc;       // planes per z-chunk (a multiple of 4)
  int ntx, nty, nzc, nitems;  // tiles per axis, z-chunks, gas-phase work items (tile x chunk)
  int n1items;  // dielectric-phase work items: the items whose boxes hold dielectric unknowns
  int par;      // 0: x holds the iterate; 1: alt does (this CTA's copy, flipped per sweep)
  T* alt[2];    // the second buffer per phase
  const void* maps;    // 7 tensor maps (128 bytes each): x[buf][phase] (buf 0 = x, 1 = alt), b[phase], flags
  const int* list1;    // [n1items] item indices of the dielectric-phase items
  // per pass kind (0: sweep, 1: residual + restriction) a ticket counter
  // handing out the pass's items and a count of the CTAs done with it; both
  // zero between passes (the last CTA done resets them)
  int* tick;    // [4]: ticket 0, done 0, ticket 1, done 1
};

template <class T>
struct Hier {
  int nlev;  // multigrid levels
  int lc;    // first level handled inside CTA 0
  int nu1, nu2;
  int bm;       // order of the bottom inverse (0: relax the bottom instead)
  int bsweeps;  // relaxation sweeps when bm == 0
  int smem;     // 1: levels lc.. keep x, b, flags and row scratch in CTA 0's shared memory
  int gbot;     // 1: the bottom is a grid phase, a row-major dense inverse applied one warp per row
  int gkry;     // 1: the bottom is a grid phase, BiCGStab over the whole grid (no inverse, > 4096 cells)
  int kry_iters;     // its iteration cap
  T* kry;            // its vectors: 6 x [2][ncell] of the bottom level
  double* kpart;     // its per-CTA partial sums: [2 buffers][CTAs][2]
  int smem_bytes;
  const T* binv;  // [bm][bm], slot s = p * ncell + c of the coarsest level
  int off_x[MAXLEV][2], off_b[MAXLEV][2], off_f[MAXLEV], off_t[MAXLEV];  // byte offsets into shared memory
  // levels lc.. whose sparse rows are staged in shared memory too (srows = 1):
  // offsets of row_ptr, col, val, diag, irr_cell, irr_of_cell, and the entry count
  int srows[MAXLEV], off_rp[MAXLEV], off_col[MAXLEV], off_val[MAXLEV], off_dg[MAXLEV], off_ic[MAXLEV],
      off_io[MAXLEV], rnnz[MAXLEV];
  Op<T> op[MAXLEV];
  SweepLev<T> sw[MAXLEV];
};

struct Barrier {
  unsigned* count;  // arrivals, monotonically increasing over one launch (zeroed before it)
  int* err;         // set when a wait gave up
};

struct SolveCtl {
  double tol;
  int max_cycles;
  int inner;       // V-cycles per FP64 outer iteration
  int mixed;       // 1: FP32 V-cycles on the correction; 0: FP64 V-cycles on phi
  const double* bnorm;        // max |b|
  unsigned long long* norms;  // [max_cycles + 2] per-iteration residual max, zeroed by the host
  int* out;                   // [0] status, [1] outer iterations, [2] V-cycles, [3] norm slot of the final residual
  unsigned long long* trace;  // [1 + TRMAX]: count, then (code << 48 | ns) per phase of the first V-cycle
  int max_iters;              // outer iterations allowed in this launch (0: no limit); status 7 when reached
};

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier: every CTA adds one arrival to a counter that only grows and
// waits until it reaches (barriers passed) x (CTAs).  The wait is bounded by
// the SM clock: on expiry the error word is set and every CTA falls through
// (returns false) at this and every later barrier.
__device__ __forceinline__ bool grid_sync(const Barrier& B, unsigned* epoch, int gsize) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* ve = B.err;
    if (*ve == 0) {
      unsigned target = (*epoch + 1u) * (unsigned)gsize;
      *epoch += 1u;
      // the CTA's writes reach thread 0 through the block barrier and are
      // released at GPU scope by the arrival (release is cumulative); the
      // acquiring load orders the reads after the wait, and the block barrier
      // below hands that on to the other threads
      red_release_add(B.count, 1u);
      long long t0 = clock64();
      while (ld_acquire(B.count) < target) {
        if (clock64() - t0 > BAR_WAIT_CYCLES) {
          atomicOr(B.err, 1);
          break;
        }
      }
    }
  }
  __syncthreads();
  volatile int* ve = B.err;
  return *ve == 0;
}

// execution context of a phase: the whole grid, or CTA 0 alone
constexpr int TRMAX = 4096;  // phase records of the first V-cycle (diagnostics)

struct Ctx {
  long long i0, st;
  bool local;
  Barrier B;
  unsigned* epoch;         // shared-memory barrier count of this CTA
  unsigned long long* tr;  // phase trace (CTA 0 of the group, first V-cycle) or null
  unsigned* tn;            // shared-memory trace length
  int gcta, gsize;         // this CTA's index in its group and the group's CTA count
  // barrier ending a phase; `code` = (level << 4) | kind names the phase for the trace
  __device__ __forceinline__ bool sync(int code) const {
    bool ok = true;
    if (local) __syncthreads();
    else ok = grid_sync(B, epoch, gsize);
    if (tr && gcta == 0 && threadIdx.x == 0 && *tn < TRMAX) {
      tr[1 + *tn] = ((unsigned long long)code << 48) | (now_ns() & 0xffffffffffffULL);
      *tn += 1;
    }
    return ok;
  }
};


// One colour of red-black Gauss-Seidel on regular cells.  Each thread takes
// U cells a grid stride apart and issues all their loads before any store, so
// that many loads are in flight per thread (the phase is latency bound).
template <class T>
__device__ __forceinline__ void ph_dense_scalar(const Op<T>& o, int colour, const Ctx& c) {
  constexpr int U = 4;
  int hx = (o.n[0] + 1) >> 1;  // cells of one colour per x row (either parity of n0)
  long long work = (o.ncell / o.n[0]) * hx;
  for (long long t0 = c.i0; t0 < work; t0 += U * c.st) {
    long long cc[U];
    int I[U][3];
    bool act[U];
    int pp[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      long long t = t0 + u * c.st;
      act[u] = false;
      cc[u] = 0;
      pp[u] = 0;
      if (t < work) {
        unsigned tu = (unsigned)t;
        unsigned row = fdiv(tu, o.dhx);
        unsigned kq = fdiv(row, o.dn1);
        int j = (int)(row - kq * (unsigned)o.n[1]);
        int k = (int)kq;
        int i = 2 * (int)(tu - row * (unsigned)hx) + ((j + k + colour) & 1);
        I[u][0] = i;
        I[u][1] = j;
        I[u][2] = k;
        if (i < o.n[0]) {
          cc[u] = (long long)i + (long long)o.n[0] * row;
          uint8_t f = o.flags[cc[u]];
          act[u] = !(f & F_IRR) && (f & 3);
          pp[u] = (f & 1) ? 0 : 1;
        }
      }
    }
    T val[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      val[u] = T(0);
      if (act[u]) {
        T sum, dg;
        reg_stencil(o, o.x[pp[u]], I[u], cc[u], sum, dg);
        val[u] = (o.h2e[pp[u]] * o.b[pp[u]][cc[u]] + sum) * diag_inv(o, pp[u], dg);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (act[u]) o.x[pp[u]][cc[u]] = val[u];
  }
}

template <class T>
__device__ __forceinline__ void ld4(const T* p, T v[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  }
}

// Relaxed value of the cell at position E (0..3) of a group of four x cells,
// from the group's loaded rows; the same terms in the same order as
// reg_stencil, so the result is bitwise that of the scalar path.
template <class T, int E>
__device__ __forceinline__ T relax4(const Op<T>& o, int p, int i, int j, int k, const T xc[4], T xl, T xr,
                                    const T ym[4], const T yp[4], const T zm[4], const T zp[4], const T bv[4]) {
  T sum = T(0);
  int nf = 0;
  T wd = T(0);
  if (i > 0) {
    sum += E > 0 ? xc[E > 0 ? E - 1 : 0] : xl;
    ++nf;
  } else if (o.wr[0] != T(0)) {
    wall_term(o, 0, xc[E < 3 ? E + 1 : 3], sum, nf, wd);
  }
  if (i < o.n[0] - 1) {
    sum += E < 3 ? xc[E < 3 ? E + 1 : 3] : xr;
    ++nf;
  } else if (o.wr[1] != T(0)) {
    wall_term(o, 1, xc[E > 0 ? E - 1 : 0], sum, nf, wd);
  }
  if (j > 0) {
    sum += ym[E];
    ++nf;
  } else if (o.wr[2] != T(0)) {
    wall_term(o, 2, yp[E], sum, nf, wd);
  }
  if (j < o.n[1] - 1) {
    sum += yp[E];
    ++nf;
  } else if (o.wr[3] != T(0)) {
    wall_term(o, 3, ym[E], sum, nf, wd);
  }
  if (o.D == 3) {
    if (k > 0) {
      sum += zm[E];
      ++nf;
    } else if (o.wr[4] != T(0)) {
      wall_term(o, 4, zp[E], sum, nf, wd);
    }
    if (k < o.n[2] - 1) {
      sum += zp[E];
      ++nf;
    } else if (o.wr[5] != T(0)) {
      wall_term(o, 5, zm[E], sum, nf, wd);
    }
  }
  return (o.h2e[p] * bv[E] + sum) * diag_inv(o, p, T(nf) + wd);
}

// Relaxed value of one regular cell by the scalar stencil (a group whose two
// cells of the colour lie in different phases).
template <class T>
__device__ __noinline__ T relax1(const Op<T>& o, int q, int i, int j, int k, long long cc) {
  int I[3] = {i, j, k};
  T sum, dg;
  reg_stencil(o, o.x[q], I, cc, sum, dg);
  return (o.h2e[q] * o.b[q][cc] + sum) * diag_inv(o, q, dg);
}

// One colour on regular cells, four x cells per work item (two of the
// colour): the item's flags come in one 32-bit load and each of its rows
// (centre, y and z neighbours, right-hand side) in one 16-byte vector load.
// Needs n[0] % 4 == 0 and 16-byte aligned arrays.
template <class T>
__device__ __forceinline__ unsigned quad_flags(const Op<T>& o, long long t, long long work, unsigned nq) {
  if (t >= work) return 0u;
  const unsigned row = fdiv((unsigned)t, o.dq);
  const long long base = (long long)row * o.n[0] + 4 * (long long)((unsigned)t - row * nq);
  return *reinterpret_cast<const unsigned*>(o.flags + base);
}

template <class T>
__device__ __forceinline__ void ph_dense_vec(const Op<T>& o, int colour, const Ctx& c) {
  constexpr int U = 2;
  const int n0 = o.n[0], n1 = o.n[1], n2 = o.D == 3 ? o.n[2] : 1;
  const unsigned nq = (unsigned)n0 >> 2;
  const long long work = (o.ncell / n0) * (long long)nq;
  const long long sy = n0, sz = (long long)n0 * n1;
  // the flags of the next work items are loaded one iteration ahead, so an
  // item's rows are requested without waiting for its flags
  unsigned wnext[U];
#pragma unroll
  for (int u = 0; u < U; ++u) wnext[u] = quad_flags(o, c.i0 + u * c.st, work, nq);
  for (long long t0 = c.i0; t0 < work; t0 += U * c.st) {
    T xc[U][4], ym[U][4], yp[U][4], zm[U][4], zp[U][4], bv[U][4], xl[U], xr[U];
    unsigned fw[U], wcur[U];
    long long b0[U];
    int J[U], K[U], I0[U], S[U], P[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      wcur[u] = wnext[u];
      wnext[u] = quad_flags(o, t0 + (U + u) * c.st, work, nq);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      fw[u] = 0u;
      b0[u] = 0;
      J[u] = K[u] = I0[u] = S[u] = P[u] = 0;
      xl[u] = xr[u] = T(0);
#pragma unroll
      for (int e = 0; e < 4; ++e) xc[u][e] = ym[u][e] = yp[u][e] = zm[u][e] = zp[u][e] = bv[u][e] = T(0);
      const long long t = t0 + u * c.st;
      if (t >= work) continue;
      const unsigned tu = (unsigned)t;
      const unsigned row = fdiv(tu, o.dq);
      const unsigned kq = fdiv(row, o.dn1);
      const int j = (int)(row - kq * (unsigned)n1), k = (int)kq;
      const int i0 = 4 * (int)(tu - row * nq);
      const int sh = (j + k + colour) & 1;
      const long long base = (long long)row * n0 + i0;
      const unsigned w = wcur[u];
      const unsigned fa = (w >> (8 * sh)) & 0xffu, fb = (w >> (8 * (sh + 2))) & 0xffu;
      const bool aa = !(fa & F_IRR) && (fa & 3), ab = !(fb & F_IRR) && (fb & 3);
      if (!aa && !ab) continue;
      const int p = aa ? ((fa & 1) ? 0 : 1) : ((fb & 1) ? 0 : 1);
      fw[u] = w;
      b0[u] = base;
      J[u] = j;
      K[u] = k;
      I0[u] = i0;
      S[u] = sh;
      P[u] = p;
      const T* X = o.x[p];
      ld4(X + base, xc[u]);
      if (sh == 0 && i0 > 0) xl[u] = X[base - 1];
      if (sh == 1 && i0 + 4 < n0) xr[u] = X[base + 4];
      if (j > 0) ld4(X + base - sy, ym[u]);
      if (j < n1 - 1) ld4(X + base + sy, yp[u]);
      if (o.D == 3) {
        if (k > 0) ld4(X + base - sz, zm[u]);
        if (k < n2 - 1) ld4(X + base + sz, zp[u]);
      }
      ld4(o.b[p] + base, bv[u]);
    }
    T v[U][2];
    int q[U][2];
    bool act[U][2];
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const unsigned f = (fw[u] >> (8 * (S[u] + 2 * h))) & 0xffu;
        act[u][h] = !(f & F_IRR) && (f & 3);
        q[u][h] = (f & 1) ? 0 : 1;
        v[u][h] = T(0);
      }
      if (!act[u][0] && !act[u][1]) continue;
      const int i = I0[u] + S[u];
      if (S[u] == 0) {
        if (act[u][0] && q[u][0] == P[u])
          v[u][0] = relax4<T, 0>(o, P[u], i, J[u], K[u], xc[u], xl[u], xr[u], ym[u], yp[u], zm[u], zp[u], bv[u]);
        if (act[u][1] && q[u][1] == P[u])
          v[u][1] = relax4<T, 2>(o, P[u], i + 2, J[u], K[u], xc[u], xl[u], xr[u], ym[u], yp[u], zm[u], zp[u], bv[u]);
      } else {
        if (act[u][0] && q[u][0] == P[u])
          v[u][0] = relax4<T, 1>(o, P[u], i, J[u], K[u], xc[u], xl[u], xr[u], ym[u], yp[u], zm[u], zp[u], bv[u]);
        if (act[u][1] && q[u][1] == P[u])
          v[u][1] = relax4<T, 3>(o, P[u], i + 2, J[u], K[u], xc[u], xl[u], xr[u], ym[u], yp[u], zm[u], zp[u], bv[u]);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (act[u][h] && q[u][h] != P[u]) v[u][h] = relax1(o, q[u][h], i + 2 * h, J[u], K[u], b0[u] + S[u] + 2 * h);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (act[u][h]) o.x[q[u][h]][b0[u] + S[u] + 2 * h] = v[u][h];
  }
}

template <class T>
__device__ __forceinline__ bool vec_ok(const Op<T>& o) {
  if (o.n[0] & 3) return false;
  unsigned long long a = (unsigned long long)o.flags & 3ull;
  for (int p = 0; p < 2; ++p) {
    a |= (unsigned long long)o.x[p] & 15ull;
    a |= (unsigned long long)o.b[p] & 15ull;
  }
  return a == 0;
}

template <class T>
__device__ __forceinline__ void ph_dense(const Op<T>& o, int colour, const Ctx& c) {
  if (vec_ok(o)) ph_dense_vec(o, colour, c);
  else ph_dense_scalar(o, colour, c);
}

// sparse rows [rb, re), one warp per row (lanes over the entries, then a
// shuffle reduction): mode 0 writes the Gauss-Seidel value, mode 1 the
// residual, into tmp.  Warps of the grid are interleaved over the CTAs so a
// few hundred rows still spread over every SM.
template <class T>
__device__ __forceinline__ void ph_rows(const Op<T>& o, long long rb, long long re, int mode, const Ctx& c) {
  if (c.local) {  // inside one CTA: a thread per row keeps every warp busy
    for (long long r = rb + threadIdx.x; r < re; r += blockDim.x) {
      double d = o.diag[r];
      if (d == 0.0) continue;
      long long cell = o.irr_cell[r >> 1];
      int p = (int)(r & 1);
      if constexpr (sizeof(T) == 4) {  // the FP32 V-cycle: rows in FP32 on its one-SM levels
        const T v = o.b[p][cell] - row_dot_t(o, r);
        o.tmp[r] = mode == 0 ? v / (T)d : v - (T)d * o.x[p][cell];
      } else {
        double v = (double)o.b[p][cell] - row_dot(o, r);
        o.tmp[r] = mode == 0 ? (T)(v / d) : (T)(v - d * (double)o.x[p][cell]);
      }
    }
    return;
  }
  // a group of 8 lanes per row, four rows per warp in flight: a row's cost
  // is a chain of dependent loads (descriptors, entries, gathered x), so
  // rows overlap rather than lanes splitting one row's few entries.  Lane
  // g of a group takes the row's entries e0 + g, e0 + g + 8, ... and the
  // group sums them in a fixed order, whatever warp takes the row.
  constexpr int GL = 8;
  const int g = threadIdx.x & (GL - 1);
  const long long grp = threadIdx.x / GL, ngrp = blockDim.x / GL;
  const long long w0 = grp * c.gsize + c.gcta, ws = (long long)c.gsize * ngrp;
  const unsigned gmask = 0xffu << (threadIdx.x & 24);
  const long long rend = rb + ((re - rb + ws - 1) / ws) * ws;  // every lane of a warp runs the same trips
  for (long long r = rb + w0; r < rend; r += ws) {
    const bool live = r < re;
    // the row's descriptors in one round of independent loads, then its
    // entries together with the cell's own b and x, then the gathered x
    const double d = live ? o.diag[r] : 0.0;
    const int e0 = live ? o.row_ptr[r] : 0, e1 = live ? o.row_ptr[r + 1] : 0;
    const long long cell = live ? o.irr_cell[r >> 1] : 0;
    const bool act = d != 0.0;
    const int p = (int)(r & 1);
    double bc = 0.0, xc = 0.0, s = 0.0;
    if (act) {
      bc = (double)o.b[p][cell];
      xc = (double)o.x[p][cell];
      for (int e = e0 + g; e < e1; e += GL) {
        unsigned cl = (unsigned)o.col[e];
        s += o.val[e] * (double)o.x[cl >> 30][cl & 0x3fffffffu];
      }
    }
    for (int off = GL / 2; off > 0; off >>= 1) s += __shfl_xor_sync(gmask, s, off);
    if (act && g == 0) {
      double v = bc - s;
      o.tmp[r] = mode == 0 ? (T)(v / d) : (T)(v - d * xc);
    }
  }
}

template <class T>
__device__ __forceinline__ void ph_write(const Op<T>& o, long long rb, long long re, const Ctx& c) {
  for (long long r = rb + c.i0; r < re; r += c.st) {
    const double d = o.diag[r];
    const long long cell = o.irr_cell[r >> 1];
    const T v = o.tmp[r];
    if (d != 0.0) o.x[r & 1][cell] = v;
  }
}

}  // namespace ebp
#include "sweep3d.cuh"
namespace ebp {

// Residual + restriction by blocks: one coarse cell per work item; the
// children and their face neighbours (4 x 4 without corners in 2D, the 2^3
// block and its 24 face neighbours in 3D) are loaded in one round for each
// phase the children carry, then every regular child's residual is formed with
// the terms and order of cell_residual; cut children take their sparse
// residual.  Needs fine n = 2 coarse n per axis.
template <class T, int D>
__device__ __forceinline__ void ph_restrict_blk(const Op<T>& f, const Op<T>& co, const Ctx& c) {
  constexpr int NCH = 1 << D, NP = D == 3 ? 64 : 16;
  // offsets within a coarse cell's children and their face halo fit in an
  // int: 32-bit offsets from the first child keep the registers down
  const int st[3] = {1, f.n[0], f.n[0] * f.n[1]};
  const T scale = T(1) / T(NCH);
  for (long long C = c.i0; C < co.ncell; C += c.st) {
    int IC[3];
    ijk(co, C, IC);
    if (D == 2) IC[2] = 0;
    const int O[3] = {2 * IC[0], 2 * IC[1], 2 * IC[2]};
    const long long c0 = O[0] + (long long)st[1] * O[1] + (long long)st[2] * O[2];
    const uint8_t* const fl0 = f.flags + c0;
    unsigned fl[NCH];
    unsigned any = 0u;
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
      fl[k] = fl0[(k & 1) + st[1] * ((k >> 1) & 1) + (D == 3 ? st[2] * ((k >> 2) & 1) : 0)];
      any |= fl[k];
    }
    const unsigned cfl = co.flags[C];
    T acc[2] = {T(0), T(0)};
    for (int q = 0; q < 2; ++q) {
      if (!((any >> q) & 1u)) continue;
      const T* x = f.x[q] + c0;
      const T* bq = f.b[q] + c0;
      // patch value at local offset (u, v, w) in -1..2, loaded where it lies in the grid
      T P[NP];
      T bv[NCH];
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        const int u = m % 4 - 1, v = (m / 4) % 4 - 1, w = D == 3 ? m / 16 - 1 : 0;
        const int out = (u < 0 || u > 1) + (v < 0 || v > 1) + (w < 0 || w > 1);
        P[m] = T(0);
        if (out > 1) continue;  // corners and edges are never needed
        const bool in = O[0] + u >= 0 && O[0] + u < f.n[0] && O[1] + v >= 0 && O[1] + v < f.n[1] &&
                        (D == 2 || (O[2] + w >= 0 && O[2] + w < f.n[2]));
        if (in) P[m] = x[u + st[1] * v + st[2] * w];
      }
#pragma unroll
      for (int k = 0; k < NCH; ++k) {
        const int ck = (k & 1) + st[1] * ((k >> 1) & 1) + (D == 3 ? st[2] * ((k >> 2) & 1) : 0);
        bv[k] = (((fl[k] >> q) & 1u) && !(fl[k] & F_IRR)) ? bq[ck] : T(0);
      }
#pragma unroll
      for (int k = 0; k < NCH; ++k) {
        if (!((fl[k] >> q) & 1u)) continue;
        const int ku = k & 1, kv = (k >> 1) & 1, kw = (k >> 2) & 1;
        const int I[3] = {O[0] + ku, O[1] + kv, O[2] + kw};
        const int loc[3] = {ku, kv, kw};
        if (fl[k] & F_IRR) {
          const long long cc = c0 + ku + st[1] * kv + (D == 3 ? st[2] * kw : 0);
          acc[q] += f.tmp[2 * (long long)f.irr_of_cell[cc] + q];
          continue;
        }
#define EBP_PIX(du, dv, dw) (((ku) + (du) + 1) + 4 * ((kv) + (dv) + 1) + 16 * ((kw) + (dw) + 1))
        T sum = T(0), wd = T(0);
        int nf = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const int e0 = a == 0, e1 = a == 1, e2 = a == 2;
          const T lo = P[D == 3 ? EBP_PIX(-e0, -e1, -e2) : EBP_PIX(-e0, -e1, 0) - 16];
          const T hi = P[D == 3 ? EBP_PIX(e0, e1, e2) : EBP_PIX(e0, e1, 0) - 16];
          if (I[a] > 0) {
            sum += lo;
            ++nf;
          } else if (f.wr[2 * a] != T(0)) {
            wall_term(f, 2 * a, hi, sum, nf, wd);
          }
          if (I[a] < f.n[a] - 1) {
            sum += hi;
            ++nf;
          } else if (f.wr[2 * a + 1] != T(0)) {
            wall_term(f, 2 * a + 1, lo, sum, nf, wd);
          }
        }
        const T xc = P[D == 3 ? EBP_PIX(0, 0, 0) : EBP_PIX(0, 0, 0) - 16];
#undef EBP_PIX
        (void)loc;
        acc[q] += bv[k] - f.ceps[q] * ((T(nf) + wd + f.lh[q]) * xc - sum);
      }
    }
    for (int p = 0; p < 2; ++p) {
      if (co.b[p] == nullptr) continue;
      co.b[p][C] = ((cfl >> p) & 1u) ? acc[p] * scale : T(0);
      co.x[p][C] = T(0);
    }
  }
}

template <class T>
__device__ __forceinline__ void ph_restrict_pt(const Op<T>& f, const Op<T>& co, const Ctx& c);

template <class T>
__device__ __forceinline__ void ph_restrict(const Op<T>& f, const Op<T>& co, const Ctx& c) {
  bool blk = true;
  for (int a = 0; a < f.D; ++a)
    if (f.n[a] != 2 * co.n[a]) blk = false;
  if (blk) {
    if (f.D == 3) ph_restrict_blk<T, 3>(f, co, c);
    else ph_restrict_blk<T, 2>(f, co, c);
    return;
  }
  ph_restrict_pt(f, co, c);
}

template <class T>
__device__ __forceinline__ void ph_restrict_pt(const Op<T>& f, const Op<T>& co, const Ctx& c) {
  int nch = 1 << f.D;
  T scale = T(1) / T(nch);
  for (long long C = c.i0; C < co.ncell; C += c.st) {
    int IC[3];
    ijk(co, C, IC);
    T acc[2] = {T(0), T(0)};
    for (int k = 0; k < nch; ++k) {
      int I[3] = {2 * IC[0] + (k & 1), 2 * IC[1] + ((k >> 1) & 1), f.D == 3 ? 2 * IC[2] + ((k >> 2) & 1) : 0};
      long long cf = (long long)I[0] + (long long)f.n[0] * ((long long)I[1] + (long long)f.n[1] * I[2]);
      uint8_t fl = f.flags[cf];
      for (int p = 0; p < 2; ++p)
        if ((fl >> p) & 1) acc[p] += cell_residual(f, cf, p, I);
    }
    uint8_t cf = co.flags[C];
    for (int p = 0; p < 2; ++p) {
      if (co.b[p] == nullptr) continue;
      co.b[p][C] = ((cf >> p) & 1) ? acc[p] * scale : T(0);
      co.x[p][C] = T(0);
    }
  }
}

// x_fine += P x_coarse, (bi/tri)linear where all coarse cells of the
// interpolation carry an unknown of the phase, else piecewise constant; two
// fine cells per thread with their loads issued first.
template <class T>
__device__ __forceinline__ T prolong_value(const Op<T>& f, const Op<T>& co, long long C, const int sdir[3], bool inside,
                                           int p) {
  const long long st3[3] = {1, co.n[0], (long long)co.n[0] * co.n[1]};
  const int ncn = 1 << f.D;
  const T* xc = co.x[p];
  bool lin = inside;
  if (lin)
    for (int k = 1; k < ncn && lin; ++k) {
      long long n = C;
      for (int a = 0; a < f.D; ++a)
        if ((k >> a) & 1) n += sdir[a] * st3[a];
      if (!((co.flags[n] >> p) & 1)) lin = false;
    }
  if (!lin) return xc[C];
  T acc = T(0);
  for (int k = 0; k < ncn; ++k) {
    long long n = C;
    T w = T(1);
    for (int a = 0; a < f.D; ++a) {
      if ((k >> a) & 1) {
        n += sdir[a] * st3[a];
        w *= T(0.25);
      } else {
        w *= T(0.75);
      }
    }
    acc += w * xc[n];
  }
  return acc;
}

// Prolongation by blocks: one coarse cell and its 2^D children per work item.
// The coarse 3^D neighbourhood (flags, values of the phases the children
// carry) and the children's flags and values are loaded in one round; each
// child then gets the (bi/tri)linear value of prolong_value, same weights in
// the same order, or the constant one.  Needs fine n = 2 coarse n per axis.
// Neighbours and children are reached by 32-bit offsets from the cell (the
// offsets of a 3^D neighbourhood and of the children fit in an int), which
// keeps the persistent kernel's register use down (no spills with them, 64
// bytes with 64-bit indices per neighbour).
template <class T, int D>
__device__ __forceinline__ void prolong_cell(const Op<T>& f, const Op<T>& co, long long C, const int IC[3]) {
  constexpr int NB = D == 3 ? 27 : 9, NCH = 1 << D;
  const int sc1 = co.n[0], sc2 = co.n[0] * co.n[1];
  const int sf1 = f.n[0], sf2 = f.n[0] * f.n[1];
  const long long F0 = (long long)(2 * IC[0]) + (long long)sf1 * (2 * IC[1]) + (D == 3 ? (long long)sf2 * (2 * IC[2]) : 0);
  // children's flags and the coarse neighbourhood's, as one bit mask per phase
  int cf[NCH];
  unsigned fm[2] = {0u, 0u}, cm[2] = {0u, 0u};
  const uint8_t* const ffl = f.flags + F0;
#pragma unroll
  for (int k = 0; k < NCH; ++k) {
    cf[k] = (k & 1) + sf1 * ((k >> 1) & 1) + (D == 3 ? sf2 * ((k >> 2) & 1) : 0);
    const unsigned v = ffl[cf[k]];
    fm[0] |= (v & 1u) << k;
    fm[1] |= ((v >> 1) & 1u) << k;
  }
  const uint8_t* const cfl = co.flags + C;
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    const int o0 = m % 3 - 1, o1 = (m / 3) % 3 - 1, o2 = D == 3 ? m / 9 - 1 : 0;
    const bool in = IC[0] + o0 >= 0 && IC[0] + o0 < co.n[0] && IC[1] + o1 >= 0 && IC[1] + o1 < co.n[1] &&
                    (D == 2 || (IC[2] + o2 >= 0 && IC[2] + o2 < co.n[2]));
    const unsigned v = in ? cfl[o0 + o1 * sc1 + o2 * sc2] : 0u;
    cm[0] |= (v & 1u) << m;
    cm[1] |= ((v >> 1) & 1u) << m;
  }
  for (int q = 0; q < 2; ++q) {
    if (!fm[q]) continue;
    T cx[NB], xo[NCH];
    const T* const xcq = co.x[q] + C;
    T* const xfq = f.x[q] + F0;
#pragma unroll
    for (int m = 0; m < NB; ++m) {
      const int o0 = m % 3 - 1, o1 = (m / 3) % 3 - 1, o2 = D == 3 ? m / 9 - 1 : 0;
      cx[m] = ((cm[q] >> m) & 1u) ? xcq[o0 + o1 * sc1 + o2 * sc2] : T(0);
    }
#pragma unroll
    for (int k = 0; k < NCH; ++k) xo[k] = ((fm[q] >> k) & 1u) ? xfq[cf[k]] : T(0);
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
      if (!((fm[q] >> k) & 1u)) continue;
      const int sd0 = (k & 1) ? 1 : -1, sd1 = ((k >> 1) & 1) ? 1 : -1, sd2 = ((k >> 2) & 1) ? 1 : -1;
      bool lin = IC[0] + sd0 >= 0 && IC[0] + sd0 < co.n[0] && IC[1] + sd1 >= 0 && IC[1] + sd1 < co.n[1] &&
                 (D == 2 || (IC[2] + sd2 >= 0 && IC[2] + sd2 < co.n[2]));
      // neighbourhood slot of the corner whose offset bits j step sd along each axis
      const int centre = D == 3 ? 13 : 4;
#define EBP_SLOT(j) (centre + (((j) & 1) ? sd0 : 0) + ((((j) >> 1) & 1) ? 3 * sd1 : 0) + \
                     ((D == 3 && (((j) >> 2) & 1)) ? 9 * sd2 : 0))
#pragma unroll
      for (int j = 1; j < NCH; ++j)
        if (!((cm[q] >> EBP_SLOT(j)) & 1u)) lin = false;
      T add;
      if (!lin) {
        add = cx[centre];
      } else {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
          T w = T(1);
          for (int a = 0; a < D; ++a) w *= ((j >> a) & 1) ? T(0.25) : T(0.75);
          acc += w * cx[EBP_SLOT(j)];
        }
        add = acc;
      }
#undef EBP_SLOT
      xfq[cf[k]] = xo[k] + add;
    }
  }
}

template <class T, int D>
__device__ __forceinline__ void ph_prolong_blk(const Op<T>& f, const Op<T>& co, const Ctx& c) {
  for (long long C = c.i0; C < co.ncell; C += c.st) {
    int IC[3];
    ijk(co, C, IC);
    if (D == 2) IC[2] = 0;
    prolong_cell<T, D>(f, co, C, IC);
  }
}

template <class T>
__device__ __forceinline__ void ph_prolong_pt(const Op<T>& f, const Op<T>& co, const Ctx& c);

template <class T>
__device__ __forceinline__ void ph_prolong(const Op<T>& f, const Op<T>& co, const Ctx& c) {
  bool blk = true;
  for (int a = 0; a < f.D; ++a)
    if (f.n[a] != 2 * co.n[a]) blk = false;
  if (blk) {
    if (f.D == 3) ph_prolong_blk<T, 3>(f, co, c);
    else ph_prolong_blk<T, 2>(f, co, c);
    return;
  }
  ph_prolong_pt(f, co, c);
}

template <class T>
__device__ __forceinline__ void ph_prolong_pt(const Op<T>& f, const Op<T>& co, const Ctx& c) {
  constexpr int U = 2;
  for (long long c0 = c.i0; c0 < f.ncell; c0 += U * c.st) {
    T add[U][2], old[U][2];
    uint8_t fl[U];
    long long cfs[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      long long cf = c0 + u * c.st;
      cfs[u] = cf;
      fl[u] = 0;
      add[u][0] = add[u][1] = old[u][0] = old[u][1] = T(0);
      if (cf >= f.ncell) continue;
      fl[u] = f.flags[cf];
      if (!(fl[u] & 3)) continue;
      int I[3];
      ijk(f, cf, I);
      int IC[3] = {I[0] >> 1, I[1] >> 1, f.D == 3 ? I[2] >> 1 : 0};
      int sdir[3];
      bool inside = true;
      for (int a = 0; a < 3; ++a) {
        sdir[a] = (I[a] & 1) ? 1 : -1;
        if (a < f.D) {
          int nb = IC[a] + sdir[a];
          if (nb < 0 || nb >= co.n[a]) inside = false;
        }
      }
      long long C = (long long)IC[0] + (long long)co.n[0] * ((long long)IC[1] + (long long)co.n[1] * IC[2]);
      for (int q = 0; q < 2; ++q)
        if ((fl[u] >> q) & 1) {
          add[u][q] = prolong_value(f, co, C, sdir, inside, q);
          old[u][q] = f.x[q][cf];
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      for (int q = 0; q < 2; ++q)
        if ((fl[u] >> q) & 1) f.x[q][cfs[u]] = old[u][q] + add[u][q];
  }
}

// nu red-black Gauss-Seidel sweeps.  Per colour, two phases: first the
// sparse rows of the colour's cut cells get new values from the current
// iterate (into tmp; rows of one colour may couple through EB stencils, so
// none may see another's new value); then the colour's regular cells relax
// and the cut-cell values are written.  A regular cell's stencil reaches only
// cells of the other colour, so neither part of the second phase reads what
// the other writes and the result does not depend on thread timing.
template <class T>
__device__ bool ph_smooth(const Op<T>& o, int nu, const Ctx& c, int l) {
  for (int s = 0; s < nu; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      long long rb = colour == 0 ? 0 : 2 * o.nirr_red, re = colour == 0 ? 2 * o.nirr_red : 2 * o.nirr;
      if (re > rb) {
        ph_rows(o, rb, re, 0, c);
        if (!c.sync((l << 4) | 2)) return false;
        ph_write(o, rb, re, c);
      }
      ph_dense(o, colour, c);
      if (!c.sync((l << 4) | (colour ? 3 : 1))) return false;
    }
  return true;
}

// nu sweeps of grid level l: tile-streamed when the level has them (and the
// group has CTAs besides CTA 0), else the colour passes above.  A streamed
// sweep relaxes, in order, the red cut cells (their sparse rows from the
// current iterate, then written), the red and the black regular cells in one
// pass over the level, and the black cut cells.  Within each of the four
// groups no cell reads another's new value except through the colour order,
// as in the colour passes.
// SW: the kernel carries the tile-streamed passes (an instantiation without
// them keeps their out-of-line calls, and the registers those cost around
// the call sites, out of every other solve).
template <class T, bool SW>
__device__ bool ph_smooth_grid(const Hier<T>& H, int l, int nu, const Ctx& c) {
  const Op<T>& o = H.op[l];
  if (!SW || !H.sw[l].on || c.local || c.gsize < 2) return ph_smooth(o, nu, c, l);
  const long long rr = 2 * o.nirr_red, rn = 2 * o.nirr;
  for (int s = 0; s < nu; ++s) {
    if (rr > 0) {
      ph_rows(o, 0, rr, 0, c);
      if (!c.sync((l << 4) | 2)) return false;
      ph_write(o, 0, rr, c);
      if (!c.sync((l << 4) | 4)) return false;
    }
    if (!ph_sweep3d(H, l, c)) return false;
    if (!c.sync((l << 4) | 13)) return false;
    if (rn > rr) {
      ph_rows(H.op[l], rr, rn, 0, c);  // H.op[l]: the swapped view, x now the new iterate
      if (!c.sync((l << 4) | 2)) return false;
      ph_write(H.op[l], rr, rn, c);
      if (!c.sync((l << 4) | 4)) return false;
    }
  }
  return true;
}

template <class T>
__device__ bool ph_bottom(const Hier<T>& H, const Op<T>* ops, const Ctx& c) {
  const Op<T>& o = ops[H.nlev - 1];
  if (H.bm == 0) return ph_smooth(o, H.bsweeps, c, H.nlev - 1);
  long long nc = o.ncell;
  for (long long i = c.i0; i < H.bm; i += c.st) {
    int p = (int)(i / nc);
    long long cell = i - p * nc;
    if (!((o.flags[cell] >> p) & 1)) continue;
    T acc = T(0);
    for (int j = 0; j < H.bm; ++j) {  // binv is stored transposed: threads read consecutive entries
      int q = j / (int)nc;
      long long cj = j - q * nc;
      acc += H.binv[(long long)j * H.bm + i] * o.b[q][cj];
    }
    o.x[p][cell] = acc;
  }
  return c.sync(((H.nlev - 1) << 4) | 9);
}

// bottom solve over the whole grid: x = binv b with binv row-major, one warp
// per row (lanes over the columns, then a shuffle reduction)
template <class T>
__device__ bool ph_bottom_grid(const Hier<T>& H, const Ctx& c) {
  const Op<T>& o = H.op[H.nlev - 1];
  const long long nc = o.ncell;
  const int lane = threadIdx.x & 31;
  const long long w0 = (long long)(threadIdx.x >> 5) * c.gsize + c.gcta;
  const long long ws = (long long)c.gsize * (blockDim.x >> 5);
  for (long long i = w0; i < H.bm; i += ws) {
    const int p = (int)(i / nc);
    const long long cell = i - p * nc;
    if (!((o.flags[cell] >> p) & 1)) continue;
    const T* row = H.binv + i * H.bm;
    T acc = T(0);
    for (int j = lane; j < H.bm; j += 32) {
      const int q = j >= nc ? 1 : 0;
      acc += row[j] * o.b[q][j - q * nc];
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) o.x[p][cell] = acc;
  }
  return c.sync(((H.nlev - 1) << 4) | 9);
}

// levels lc.. inside CTA 0, on the shared-memory copies when H.smem
template <class T>
__device__ void coarse_part(const Hier<T>& H, const Op<T>* lop, const Ctx& L) {
  const int lc = H.lc;
  if (H.smem) {  // right-hand side of level lc in, correction zero
    const Op<T>& g = H.op[lc];
    const Op<T>& s = lop[lc];
    for (long long c = L.i0; c < g.ncell; c += L.st)
      for (int p = 0; p < 2; ++p)
        if (g.b[p]) {
          s.b[p][c] = g.b[p][c];
          s.x[p][c] = g.x[p][c];  // zero below the finest level; the iterate itself when lc == 0
        }
    __syncthreads();
  }
  for (int l = lc; l < H.nlev - 1; ++l) {
    const Op<T>& o = lop[l];
    ph_smooth(o, H.nu1, L, l);
    if (o.nirr) {
      ph_rows(o, 0, 2 * o.nirr, 1, L);
      L.sync((l << 4) | 5);
    }
    ph_restrict(o, lop[l + 1], L);
    L.sync((l << 4) | 6);
  }
  ph_bottom(H, lop, L);
  for (int l = H.nlev - 2; l >= lc; --l) {
    ph_prolong(lop[l], lop[l + 1], L);
    L.sync((l << 4) | 7);
    ph_smooth(lop[l], H.nu2, L, l);
  }
  if (H.smem) {  // correction of level lc out
    const Op<T>& g = H.op[lc];
    const Op<T>& s = lop[lc];
    for (long long c = L.i0; c < g.ncell; c += L.st)
      for (int p = 0; p < 2; ++p)
        if (g.x[p]) g.x[p][c] = s.x[p][c];
  }
}

// ---------------------------------------------------------------- Krylov bottom
// Sum over the CTA in a fixed order (tree over warps): deterministic.
__device__ __forceinline__ double cta_sum(double v) {
  __shared__ double part[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) part[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < nw; ++k) t += part[k];
  return t;
}

// Two grid-wide sums at once: each CTA stores its partials in buffer `buf`,
// the grid barrier follows, then every thread adds the partials in CTA order
// (deterministic).  Consecutive reductions alternate buffers, so a CTA never
// overwrites partials another CTA may still be reading.
__device__ __forceinline__ bool grid_sum2(double* kpart, int buf, double a, double b, const Ctx& c, int code,
                                          double& sa, double& sb) {
  a = cta_sum(a);
  b = cta_sum(b);
  double* pb = kpart + (long long)buf * 2 * c.gsize;
  if (threadIdx.x == 0) {
    pb[2 * c.gcta] = a;
    pb[2 * c.gcta + 1] = b;
  }
  if (!c.sync(code)) return false;
  // warp 0 reads the partials through L2 (lane j takes CTAs j, j + 32, ...)
  // and reduces them by a fixed shuffle tree: the same sums in every CTA
  __shared__ double res[2];
  if (threadIdx.x < 32) {
    double ta = 0.0, tb = 0.0;
    for (int k = threadIdx.x; k < c.gsize; k += 32) {
      ta += __ldcg(pb + 2 * k);
      tb += __ldcg(pb + 2 * k + 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
      ta += __shfl_xor_sync(0xffffffffu, ta, o);
      tb += __shfl_xor_sync(0xffffffffu, tb, o);
    }
    if (threadIdx.x == 0) {
      res[0] = ta;
      res[1] = tb;
    }
  }
  __syncthreads();
  sa = res[0];
  sb = res[1];
  __syncthreads();
  return true;
}

// z = A y on the bottom level (its own operator: implicit regular stencil,
// sparse cut-cell rows; entries without an unknown 0), grid-stride over cells;
// returns this thread's partial of (w, z) and (z, z) when w is given
template <class T>
__device__ __forceinline__ void bot_matvec_grid(const Op<T>& o, const T* y, T* z, const Ctx& c) {
  const long long n = o.ncell;
  for (long long cc = c.i0; cc < n; cc += c.st) {
    const uint8_t f = o.flags[cc];
    for (int p = 0; p < 2; ++p) {
      T acc = T(0);
      if ((f >> p) & 1) {
        if (f & F_IRR) {
          const long long r = 2 * (long long)o.irr_of_cell[cc] + p;
          double a = o.diag[r] * (double)y[p * n + cc];
          for (int e = o.row_ptr[r]; e < o.row_ptr[r + 1]; ++e) {
            const unsigned cl = (unsigned)o.col[e];
            a += o.val[e] * (double)y[(long long)(cl >> 30) * n + (cl & 0x3fffffffu)];
          }
          acc = (T)a;
        } else {
          int I[3];
          ijk(o, cc, I);
          T sum, dg;
          reg_stencil(o, y + p * n, I, cc, sum, dg);
          acc = o.ceps[p] * ((dg + o.lh[p]) * y[p * n + cc] - sum);
        }
      }
      z[p * n + cc] = acc;
    }
  }
}

// BiCGStab on the bottom level over the whole grid, from x = 0, until
// |r|_2 <= 1e-3 |b|_2 or kry_iters iterations.  Every thread computes the same
// scalars from the same ordered sums, so all CTAs take the same path through
// the five grid barriers of an iteration.
template <class T>
__device__ bool ph_bicgstab_grid(const Hier<T>& H, const Ctx& c) {
  const int code = ((H.nlev - 1) << 4) | 9;
  const Op<T>& o = H.op[H.nlev - 1];
  if (c.gsize > 1024) return ph_smooth(o, H.bsweeps, c, H.nlev - 1);  // partial sums sized for 1024 CTAs
  const long long n = o.ncell, m = 2 * n;
  T *r = H.kry, *r0 = r + m, *pv = r0 + m, *v = pv + m, *sv = v + m, *t = sv + m;
  int buf = 0;
  double la = 0.0, lb = 0.0;
  for (long long cc = c.i0; cc < n; cc += c.st) {
    const uint8_t f = o.flags[cc];
    for (int p = 0; p < 2; ++p) {
      const long long i = p * n + cc;
      const T bi = (((f >> p) & 1) && o.b[p]) ? o.b[p][cc] : T(0);
      r[i] = r0[i] = bi;
      pv[i] = v[i] = T(0);
      if (o.x[p]) o.x[p][cc] = T(0);
      la += (double)bi * (double)bi;
    }
  }
  double bb = 0.0, rho1 = 0.0;
  if (!grid_sum2(H.kpart, buf, la, la, c, code, bb, rho1)) return false;
  buf ^= 1;
  if (!(bb > 0.0)) return true;
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  for (int it = 0; it < H.kry_iters; ++it) {
    if (rho1 == 0.0 || omega == 0.0) break;
    const double beta = (rho1 / rho) * (alpha / omega);
    for (long long i = c.i0; i < m; i += c.st) pv[i] = (T)((double)r[i] + beta * ((double)pv[i] - omega * (double)v[i]));
    if (!c.sync(code)) return false;
    bot_matvec_grid(o, pv, v, c);
    la = 0.0;
    for (long long cc = c.i0; cc < n; cc += c.st)
      for (int p = 0; p < 2; ++p) la += (double)r0[p * n + cc] * (double)v[p * n + cc];
    double rv = 0.0, dummy = 0.0;
    if (!grid_sum2(H.kpart, buf, la, 0.0, c, code, rv, dummy)) return false;
    buf ^= 1;
    if (rv == 0.0) break;
    alpha = rho1 / rv;
    for (long long i = c.i0; i < m; i += c.st) sv[i] = (T)((double)r[i] - alpha * (double)v[i]);
    if (!c.sync(code)) return false;
    bot_matvec_grid(o, sv, t, c);
    la = lb = 0.0;
    for (long long cc = c.i0; cc < n; cc += c.st)
      for (int p = 0; p < 2; ++p) {
        const double tv = (double)t[p * n + cc];
        la += tv * (double)sv[p * n + cc];
        lb += tv * tv;
      }
    double ts = 0.0, tt = 0.0;
    if (!grid_sum2(H.kpart, buf, la, lb, c, code, ts, tt)) return false;
    buf ^= 1;
    omega = tt > 0.0 ? ts / tt : 0.0;
    la = lb = 0.0;
    for (long long i = c.i0; i < m; i += c.st) {
      const int p = (int)(i / n);
      const long long cc = i - p * n;
      if (o.x[p] && ((o.flags[cc] >> p) & 1))
        o.x[p][cc] = (T)((double)o.x[p][cc] + alpha * (double)pv[i] + omega * (double)sv[i]);
      const double ri = (double)sv[i] - omega * (double)t[i];
      r[i] = (T)ri;
      la += (double)r0[i] * ri;
      lb += ri * ri;
    }
    double rho_next = 0.0, rr = 0.0;
    if (!grid_sum2(H.kpart, buf, la, lb, c, code, rho_next, rr)) return false;
    buf ^= 1;
    rho = rho1;
    rho1 = rho_next;
    if (rr <= 1e-6 * bb) break;
  }
  return true;
}

template <class T, bool SW>
__device__ bool vcycle_dev(const Hier<T>& H, const Op<T>* lop, const Ctx& G) {
  for (int l = 0; l < H.lc; ++l) {
    const Op<T>& o = H.op[l];
    if (!ph_smooth_grid<T, SW>(H, l, H.nu1, G)) return false;
    if (o.nirr) {
      ph_rows(o, 0, 2 * o.nirr, 1, G);
      if (!G.sync((l << 4) | 5)) return false;
    }
    if (SW && H.sw[l].on && H.sw[l].rs && G.gsize >= 2 && o.n[0] == 2 * H.op[l + 1].n[0] && o.n[1] == 2 * H.op[l + 1].n[1] &&
        o.n[2] == 2 * H.op[l + 1].n[2]) {
      if (!ph_restrict3d(H, l, G)) return false;
    } else {
      ph_restrict(o, H.op[l + 1], G);
    }
    if (!G.sync((l << 4) | 6)) return false;
  }
  if (H.gbot) {
    if (!ph_bottom_grid(H, G)) return false;
  } else if (H.gkry) {
    if (!ph_bicgstab_grid(H, G)) return false;
    if (!G.sync(((H.nlev - 1) << 4) | 9)) return false;
  } else {
    if (G.gcta == 0) {
      Ctx L{(long long)threadIdx.x, (long long)blockDim.x, true, G.B, G.epoch, G.tr, G.tn, 0, 1};
      coarse_part(H, lop, L);
    }
    if (!G.sync((15 << 4) | 8)) return false;
  }
  for (int l = H.lc - 1; l >= 0; --l) {
    ph_prolong(H.op[l], H.op[l + 1], G);
    if (!G.sync((l << 4) | 7)) return false;
    if (!ph_smooth_grid<T, SW>(H, l, H.nu2, G)) return false;
  }
  return true;
}

// FP64 residual of the finest level and its max norm into norms[slot]; in
// mixed mode it also becomes the FP32 inner right-hand side (correction zeroed)
template <class T>
__device__ bool ph_resid64(const Op<double>& o, const Hier<T>& H, int mixed, unsigned long long* norm,
                           const Ctx& G) {
  if (o.nirr) {
    ph_rows(o, 0, 2 * o.nirr, 1, G);
    if (!G.sync((14 << 4) | 10)) return false;
  }
  double mx = 0.0;
  const Op<T>& inner = H.op[0];
  for (long long cc = G.i0; cc < o.ncell; cc += G.st) {
    uint8_t f = o.flags[cc];
    int I[3];
    ijk(o, cc, I);
    for (int p = 0; p < 2; ++p) {
      double r = 0.0;
      if ((f >> p) & 1) r = cell_residual(o, cc, p, I);
      mx = fmax(mx, fabs(r));
      if (mixed && inner.b[p]) {
        inner.b[p][cc] = (T)r;
        inner.x[p][cc] = T(0);
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(norm, (unsigned long long)__double_as_longlong(mx));
  return G.sync((14 << 4) | 11);
}

template <class T>
__device__ void ph_update64(const Op<double>& o, const Op<T>& inner, const Ctx& G) {
  for (long long cc = G.i0; cc < o.ncell; cc += G.st) {
    uint8_t f = o.flags[cc];
    if (f & 1) o.x[0][cc] += (double)inner.x[0][cc];
    if ((f & 2) && inner.x[1]) o.x[1][cc] += (double)inner.x[1][cc];
  }
}

__device__ __forceinline__ double load_norm(const unsigned long long* p) {
  volatile const unsigned long long* vp = p;
  return __longlong_as_double((long long)*vp);
}

// The solve: residual, test, (inner V-cycles, update)*, until converged or capped.
// copy of `words` 4-byte words from global into shared memory by the whole CTA
__device__ __forceinline__ void stage_words(unsigned char* dst, const void* src, long long words) {
  const int* s = (const int*)src;
  int* d = (int*)dst;
  for (long long i = threadIdx.x; i < words; i += blockDim.x) d[i] = s[i];
}

// The V-cycle as the FP64 solve calls it: out of line, which keeps ptxas
// from spilling the FP64 V-cycle's registers into the outer loop (1276 bytes
// of spills inlined, 92 out of line); the FP32 V-cycle stays inline (64
// bytes inlined, 92 out of line).
template <class T, bool SW>
__device__ __noinline__ bool vcycle_dev_ool(const Hier<T>& H, const Op<T>* lop, const Ctx& G) {
  return vcycle_dev<T, SW>(H, lop, G);
}
template <class T, bool SW>
__device__ __forceinline__ bool vcycle_call(const Hier<T>& H, const Op<T>* lop, const Ctx& G) {
  if constexpr (sizeof(T) == 8) return vcycle_dev_ool<T, SW>(H, lop, G);
  else return vcycle_dev<T, SW>(H, lop, G);
}

template <class T, bool SW>
__device__ __forceinline__ void solve_group(const Hier<T>* __restrict__ Hg, const Op<double>* __restrict__ Fg,
                                            const SolveCtl& ctl, const Barrier& B, int gcta, int gsize) {
  __shared__ Hier<T> H;
  __shared__ Op<double> F;
  __shared__ Op<T> lop[MAXLEV];  // level views used inside CTA 0 (shared-memory data for levels lc..)
  __shared__ unsigned epoch;
  __shared__ unsigned tn;
  extern __shared__ __align__(128) unsigned char dyn[];
  {
    const int* src = (const int*)Hg;
    int* dst = (int*)&H;
    for (int i = threadIdx.x; i < (int)(sizeof(Hier<T>) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    const int* s2 = (const int*)Fg;
    int* d2 = (int*)&F;
    for (int i = threadIdx.x; i < (int)(sizeof(Op<double>) / sizeof(int)); i += blockDim.x) d2[i] = s2[i];
    if (threadIdx.x == 0) {
      epoch = 0u;
      tn = 0u;
    }
  }
  __syncthreads();
  if (gcta == 0) {
    if (threadIdx.x < MAXLEV && (int)threadIdx.x < H.nlev) {
      int l = threadIdx.x;
      Op<T> v = H.op[l];
      if (H.smem && l >= H.lc) {
        for (int p = 0; p < 2; ++p) {
          v.x[p] = v.x[p] ? (T*)(dyn + H.off_x[l][p]) : nullptr;
          v.b[p] = v.b[p] ? (T*)(dyn + H.off_b[l][p]) : nullptr;
        }
        v.flags = (const uint8_t*)(dyn + H.off_f[l]);
        v.tmp = (T*)(dyn + H.off_t[l]);
        if (H.srows[l]) {
          v.row_ptr = (const int*)(dyn + H.off_rp[l]);
          v.col = (const int*)(dyn + H.off_col[l]);
          v.val = (const double*)(dyn + H.off_val[l]);
          v.diag = (const double*)(dyn + H.off_dg[l]);
          v.irr_cell = (const int*)(dyn + H.off_ic[l]);
          v.irr_of_cell = (const int*)(dyn + H.off_io[l]);
        }
      }
      lop[l] = v;
    }
    if (H.smem)
      for (int l = H.lc; l < H.nlev; ++l) {
        const Op<T>& g = H.op[l];
        for (long long c = threadIdx.x; c < g.ncell; c += blockDim.x) dyn[H.off_f[l] + c] = g.flags[c];
        if (H.srows[l]) {  // the level's rows are constant over the launch: staged once
          const long long nr = 2 * g.nirr;
          stage_words(dyn + H.off_rp[l], g.row_ptr, nr + 1);
          stage_words(dyn + H.off_col[l], g.col, H.rnnz[l]);
          stage_words(dyn + H.off_val[l], g.val, 2 * (long long)H.rnnz[l]);
          stage_words(dyn + H.off_dg[l], g.diag, 2 * nr);
          stage_words(dyn + H.off_ic[l], g.irr_cell, g.nirr);
          stage_words(dyn + H.off_io[l], g.irr_of_cell, g.ncell);
        }
      }
  }
  __syncthreads();
  // warps of the grid interleaved over the CTAs: lanes stay on consecutive
  // elements (coalesced) while consecutive 32-element chunks land on different SMs
  const long long gi = ((long long)(threadIdx.x >> 5) * gsize + gcta) * 32 + (threadIdx.x & 31);
  Ctx G{gi, (long long)gsize * blockDim.x, false, B, &epoch, nullptr, &tn, gcta, gsize};
  const double bn = *ctl.bnorm;
  int it = 0, cycles = 0, status = 0;
  double r0 = 0.0, r = 0.0;
  if (bn == 0.0) {  // b = 0: the solution is 0
    for (long long cc = G.i0; cc < F.ncell; cc += G.st) {
      F.x[0][cc] = 0.0;
      if (F.x[1]) F.x[1][cc] = 0.0;
    }
  }
  for (; bn != 0.0;) {
    if (!ph_resid64(F, H, ctl.mixed, ctl.norms + it, G)) {
      status = 5;
      break;
    }
    r = load_norm(ctl.norms + it);
    if (it == 0) r0 = r;
    if (r <= ctl.tol * bn) break;
    if (cycles + ctl.inner > ctl.max_cycles || !(r == r) || r > 1e6 * r0) {
      status = 3;
      break;
    }
    if (ctl.max_iters && it >= ctl.max_iters) {  // resumable: stop at a V-cycle boundary
      status = 7;
      break;
    }
    bool ok = true;
    for (int k = 0; k < ctl.inner && ok; ++k) {
      Ctx Gk = G;
      if (it == 0 && k == 0 && ctl.trace) {  // trace the first V-cycle
        Gk.tr = ctl.trace;
        if (gcta == 0 && threadIdx.x == 0) ctl.trace[1 + tn++] = ((unsigned long long)0xfff << 48) | (now_ns() & 0xffffffffffffULL);
      }
      ok = vcycle_call<T, SW>(H, lop, Gk);
    }
    if (ok && ctl.mixed) {
      ph_update64(F, H.op[0], G);
      ok = G.sync((14 << 4) | 12);
    }
    if (!ok) {
      status = 5;
      break;
    }
    cycles += ctl.inner;
    ++it;
  }
  if (gcta == 0 && threadIdx.x == 0) {
    if (ctl.trace) ctl.trace[0] = tn;
    ctl.norms[ctl.max_cycles + 1] = (unsigned long long)__double_as_longlong(r);  // final residual max
    ctl.out[0] = status;
    ctl.out[1] = it;
    ctl.out[2] = cycles;
    ctl.out[3] = it;
  }
}

template <class T, bool SW>
__global__ void __launch_bounds__(PT, 1) k_solve(const Hier<T>* __restrict__ Hg, const Op<double>* __restrict__ Fg,
                                                 SolveCtl ctl, Barrier B) {
  solve_group<T, SW>(Hg, Fg, ctl, B, (int)blockIdx.x, (int)gridDim.x);
}

// one instance of a batched solve: its hierarchy, fine operator, controls,
// barrier and the block of CTAs [start, start + size) that works on it
template <class T>
struct BatchItem {
  const Hier<T>* H;
  const Op<double>* F;
  SolveCtl ctl;
  Barrier B;
  int start, size;
};

// Many independent solves in one cooperative launch: each CTA finds its
// instance and runs the solve with the instance's own group barrier.
template <class T, bool SW>
__global__ void __launch_bounds__(PT, 1) k_solve_batch(const BatchItem<T>* __restrict__ items,
                                                       const int* __restrict__ cta_item) {
  const BatchItem<T>& it = items[cta_item[blockIdx.x]];
  solve_group<T, SW>(it.H, it.F, it.ctl, it.B, (int)blockIdx.x - it.start, it.size);
}

// Setup of the tile-streamed passes: one CTA per (tile, plane).  Entry
// t * n2 + z of has1 is set when the tile's box (the tile with the halo) holds
// a dielectric unknown in fine plane z; entry ntiles * n2 + t * cn2 + z when
// the coarse cells under the tile do in coarse plane z (cflags of the level
// below, may be null).  The host ORs the planes of each item from these.
__global__ void k_sweep_has1(const uint8_t* __restrict__ flags, int n0, int n1, int n2, int ntx, int nty,
                             const uint8_t* __restrict__ cflags, int cn0, int cn1, int cn2, uint8_t* has1) {
  const int ntiles = ntx * nty;
  const long long nfine = (long long)ntiles * n2;
  const long long b = blockIdx.x;
  int found = 0;
  if (b < nfine) {
    const int t = (int)(b / n2), z = (int)(b % n2);
    const int x0 = (t % ntx) * SW_TX, y0 = (t / ntx) * SW_TY;
    const int xa = max(x0 - SW_HX, 0), xb = min(x0 + SW_TX + SW_HX, n0);
    const int ya = max(y0 - SW_HY, 0), yb = min(y0 + SW_TY + SW_HY, n1);
    const int nx = xb - xa, ny = yb - ya;
    for (int e = threadIdx.x; e < nx * ny && !found; e += blockDim.x)
      if (flags[((long long)z * n1 + ya + e / nx) * n0 + xa + e % nx] & 2) found = 1;
  } else if (cflags) {
    const long long r = b - nfine;
    const int t = (int)(r / cn2), z = (int)(r % cn2);
    const int x0 = (t % ntx) * SW_TX, y0 = (t / ntx) * SW_TY;
    const int cxa = x0 / 2, cxb = min((x0 + SW_TX) / 2, cn0), cya = y0 / 2, cyb = min((y0 + SW_TY) / 2, cn1);
    const int mx = max(cxb - cxa, 0), my = max(cyb - cya, 0);
    for (int e = threadIdx.x; e < mx * my && !found; e += blockDim.x)
      if (cflags[((long long)z * cn1 + cya + e / mx) * cn0 + cxa + e % mx] & 2) found = 1;
  }
  if (__syncthreads_or(found) && threadIdx.x == 0) has1[b] = 1;
}

// ------------------------------------------------------------ bottom inverse

// dense matrix of the coarsest level over slots s = p * ncell + c; rows of
// slots without an unknown are identity rows
template <class T>
__global__ void k_bottom_matrix(Op<T> o, double ceps0, double ceps1, int m, double* M) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  long long nc = o.ncell;
  int p = (int)(i / nc);
  long long c = i - p * nc;
  double* row = M + i * m;  // zeroed by the caller
  uint8_t f = o.flags[c];
  if (!((f >> p) & 1)) {
    row[i] = 1.0;
    return;
  }
  if (f & F_IRR) {
    long long r = 2 * (long long)o.irr_of_cell[c] + p;
    row[i] += o.diag[r];
    for (int e = o.row_ptr[r]; e < o.row_ptr[r + 1]; ++e) {
      unsigned cl = (unsigned)o.col[e];
      long long j = (long long)(cl >> 30) * nc + (cl & 0x3fffffffu);
      row[j] += o.val[e];
    }
    return;
  }
  double ce = p ? ceps1 : ceps0;
  int I[3];
  ijk(o, c, I);
  long long st = 1;
  row[i] += ce * (double)o.lh[p];  // the Helmholtz shift
  for (int a = 0; a < o.D; ++a) {
    const double wl = (double)o.wr[2 * a], wh = (double)o.wr[2 * a + 1];
    if (I[a] > 0) {
      row[i - st] -= ce;
      row[i] += ce;
    } else if (wl != 0.0) {
      row[i + st] -= wl * ce / 3.0;
      row[i] += 3.0 * wl * ce;
    }
    if (I[a] < o.n[a] - 1) {
      row[i + st] -= ce;
      row[i] += ce;
    } else if (wh != 0.0) {
      row[i - st] -= wh * ce / 3.0;
      row[i] += 3.0 * wh * ce;
    }
    st *= o.n[a];
  }
}

// Gauss-Jordan inversion with partial pivoting by one CTA: A (m x m) is
// destroyed, Ainv receives the inverse; status[0] = 1 when a pivot vanishes.
__global__ void k_gauss_jordan(double* A, double* Ainv, int m, int* status) {
  __shared__ double sv[1024];
  __shared__ int si[1024];
  __shared__ int piv;
  __shared__ double pval;
  for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) Ainv[e] = (e / m == e % m) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    double best = -1.0;
    int bi = k;
    for (int r = k + threadIdx.x; r < m; r += blockDim.x) {
      double v = fabs(A[(long long)r * m + k]);
      if (v > best) {
        best = v;
        bi = r;
      }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) {
        double a = sv[threadIdx.x], b = sv[threadIdx.x + s];
        int ia = si[threadIdx.x], ib = si[threadIdx.x + s];
        if (b > a || (b == a && ib < ia)) {
          sv[threadIdx.x] = b;
          si[threadIdx.x] = ib;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      piv = si[0];
      pval = A[(long long)si[0] * m + k];
      if (!(fabs(pval) > 1e-300)) status[0] = 1;
    }
    __syncthreads();
    if (status[0]) return;
    int pr = piv;
    if (pr != k)
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double t = A[(long long)k * m + j];
        A[(long long)k * m + j] = A[(long long)pr * m + j];
        A[(long long)pr * m + j] = t;
        t = Ainv[(long long)k * m + j];
        Ainv[(long long)k * m + j] = Ainv[(long long)pr * m + j];
        Ainv[(long long)pr * m + j] = t;
      }
    __syncthreads();
    double inv = 1.0 / pval;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      A[(long long)k * m + j] *= inv;
      Ainv[(long long)k * m + j] *= inv;
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
      int r = (int)(e / m), j = (int)(e % m);
      if (r == k) continue;
      double fct = A[(long long)r * m + k];
      if (j == k) continue;
      A[e] -= fct * A[(long long)k * m + j];
      Ainv[e] -= fct * Ainv[(long long)k * m + j];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
      if (r == k) continue;
      double fct = A[(long long)r * m + k];
      Ainv[(long long)r * m + k] -= fct * Ainv[(long long)k * m + k];
      A[(long long)r * m + k] = 0.0;
    }
    __syncthreads();
  }
}

// transpose and convert the bottom inverse (m x m)
template <class T, class S = double>
__global__ void k_convert(const S* a, T* b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long m = (long long)llrint(sqrt((double)n));
  if (i < n) b[(i % m) * m + i / m] = (T)a[i];
}

template <class T>
__global__ void k_from_float(const float* a, T* b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

__global__ void k_to_float(const double* a, float* b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// FP32 Gauss-Jordan for larger bottoms, one pivot step in two launches.
// Step k, part 1 (one CTA): partial pivoting on column k, row swap, row k
// scaled by the pivot; Ai starts as the identity.
__global__ void k_gj_pivot(float* A, float* Ai, int m, int k, int* status) {
  __shared__ float sv[1024];
  __shared__ int si[1024];
  __shared__ int piv;
  __shared__ float pval;
  if (status[0]) return;
  float best = -1.0f;
  int bi = k;
  for (int r = k + threadIdx.x; r < m; r += blockDim.x) {
    float v = fabsf(A[(long long)r * m + k]);
    if (v > best) {
      best = v;
      bi = r;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      float a = sv[threadIdx.x], b = sv[threadIdx.x + s];
      int ia = si[threadIdx.x], ib = si[threadIdx.x + s];
      if (b > a || (b == a && ib < ia)) {
        sv[threadIdx.x] = b;
        si[threadIdx.x] = ib;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    piv = si[0];
    pval = A[(long long)si[0] * m + k];
    if (!(fabsf(pval) > 1e-30f)) status[0] = 1;
  }
  __syncthreads();
  if (status[0]) return;
  const int pr = piv;
  const float inv = 1.0f / pval;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    float a = A[(long long)pr * m + j], ai = Ai[(long long)pr * m + j];
    if (pr != k) {
      A[(long long)pr * m + j] = A[(long long)k * m + j];
      Ai[(long long)pr * m + j] = Ai[(long long)k * m + j];
    }
    A[(long long)k * m + j] = a * inv;
    Ai[(long long)k * m + j] = ai * inv;
  }
}

// Step k, part 2: column k eliminated from every other row, one warp per row
// (row k is only read; each warp reads its multiplier before clearing it).
__global__ void k_gj_elim(float* A, float* Ai, int m, int k, const int* status) {
  if (status[0]) return;
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= m || r == k) return;
  const float f = A[r * m + k];
  if (f == 0.0f) return;
  const float* Ak = A + (long long)k * m;
  const float* Aik = Ai + (long long)k * m;
  float* Ar = A + r * m;
  float* Air = Ai + r * m;
  for (int j = k + 1 + lane; j < m; j += 32) Ar[j] -= f * Ak[j];
  for (int j = lane; j < m; j += 32) Air[j] -= f * Aik[j];
  __syncwarp();
  if (lane == 0) Ar[k] = 0.0f;
}

__global__ void k_identity(float* Ai, int m) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (long long)m * m) Ai[e] = (e / m == e % m) ? 1.0f : 0.0f;
}

}  // namespace ebp

namespace ebp {
// barrier microbenchmark: reps grid barriers
__global__ void __launch_bounds__(PT) k_barrier_bench(Barrier B, int reps) {
  __shared__ unsigned epoch;
  if (threadIdx.x == 0) epoch = 0u;
  __syncthreads();
  for (int i = 0; i < reps; ++i)
    if (!grid_sync(B, &epoch, (int)gridDim.x)) return;
}

// bounded-wait self-test: the CTAs wait at a grid barrier sized for one more
// CTA than was launched, so the wait can only end by its clock bound; the
// kernel then returns with the error word set
__global__ void __launch_bounds__(PT) k_barrier_expiry(Barrier B) {
  __shared__ unsigned epoch;
  if (threadIdx.x == 0) epoch = 0u;
  __syncthreads();
  grid_sync(B, &epoch, (int)gridDim.x + 1);
}

// the persistent kernel's phases launched on their own, with its grid shape,
// to time them on large levels: one colour of the regular-cell sweep, and the
// residual fused with restriction (cut-cell residual rows as left in tmp)
template <class T>
__global__ void __launch_bounds__(PT) k_dense_phase(Op<T> o, int colour) {
  Ctx c{};
  c.i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  c.st = (long long)gridDim.x * blockDim.x;
  c.gsize = (int)gridDim.x;
  c.gcta = (int)blockIdx.x;
  ph_dense(o, colour, c);
}

// one tile-streamed sweep of level l on its own, in the persistent kernel's
// grid shape (CTA 0 sits out as in the solve); x -> alt as in the solve
template <class T>
__global__ void __launch_bounds__(PT, 1) k_sweep_phase(const Hier<T>* __restrict__ Hg, int l, int* err) {
  __shared__ Hier<T> H;
  const int* src = (const int*)Hg;
  int* dst = (int*)&H;
  for (int i = threadIdx.x; i < (int)(sizeof(Hier<T>) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  Ctx c{};
  c.gsize = (int)gridDim.x;
  c.gcta = (int)blockIdx.x;
  c.B.err = err;
  ph_sweep3d(H, l, c);
}

// the streamed residual + restriction of level l on its own (cut-cell
// residual rows as left in tmp), in the persistent kernel's grid shape
template <class T>
__global__ void __launch_bounds__(PT, 1) k_restrict3d_phase(const Hier<T>* __restrict__ Hg, int l, int* err) {
  __shared__ Hier<T> H;
  const int* src = (const int*)Hg;
  int* dst = (int*)&H;
  for (int i = threadIdx.x; i < (int)(sizeof(Hier<T>) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  Ctx c{};
  c.gsize = (int)gridDim.x;
  c.gcta = (int)blockIdx.x;
  c.B.err = err;
  ph_restrict3d(H, l, c);
}

template <class T>
__global__ void __launch_bounds__(PT) k_restrict_phase(Op<T> f, Op<T> co) {
  Ctx c{};
  c.i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  c.st = (long long)gridDim.x * blockDim.x;
  c.gsize = (int)gridDim.x;
  c.gcta = (int)blockIdx.x;
  ph_restrict(f, co, c);
}

// the prolongation of level 1's correction onto level 0 (x += P e), on its own
template <class T>
__global__ void __launch_bounds__(PT) k_prolong_phase(Op<T> f, Op<T> co) {
  Ctx c{};
  c.i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  c.st = (long long)gridDim.x * blockDim.x;
  c.gsize = (int)gridDim.x;
  c.gcta = (int)blockIdx.x;
  ph_prolong(f, co, c);
}
}  // namespace ebp
