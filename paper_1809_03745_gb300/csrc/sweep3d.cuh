// sweep3d.cuh -- one red-black Gauss-Seidel sweep of a large 3D level in a
// single pass over memory (arXiv:1809.03745, Sec. 3.3.2 smooths by
// multi-colour Gauss-Seidel; the order of the colours within a sweep is a
// free choice of the multigrid, not of the discretisation).
//
// A classic colour pass reads the whole level and writes half of it, so a
// sweep moves about twice the bytes the method needs.  Here a CTA owns an
// x-y tile of 32 x 32 cells of one phase and streams it along z through
// shared memory: TMA (cp.async.bulk.tensor) brings in the tile with a halo
// of x, b and the cell flags two planes per copy, a ring of four two-plane
// slots, each copy completing an mbarrier.  Step s relaxes the red regular
// cells of two planes on the tile plus a one-cell ring (reading black values
// not yet updated), then, after one block barrier, the black regular cells
// of the two planes below (reading the new red values), and stores the two
// planes below those, final since the previous step.  The ring's red values
// equal those the neighbouring tile computes, because every read comes from
// the previous iterate: the sweep is out of place, x -> alt, and the two
// buffers swap roles afterwards.  Cut cells (sparse rows) are not touched
// here: their new values were written into x before the pass.  The regular
// cells of the two phases couple only through cut cells, so the dielectric
// phase streams in items of its own, only over the tiles that hold it.
//
// Moving two planes per step matters more than the ring depth: the pass is
// bound by the fixed cost of a pipeline step (the wait, the barrier, the
// copy issue), not by the bytes in flight.
//
// Every load and store stays inside the arrays: the TMA unit clips the boxes
// to the tensor (zero fill outside), and stores are masked to the grid.
// Waits on the mbarriers are bounded; on expiry the CTA raises the grid's
// error word, waits (bounded again) for its own copies still in flight and
// returns false.
#pragma once

namespace ebp {

// the thread layouts below: 512 threads, 16 per tile row of 32 cells (one
// colour), 32 rows; stores by 16 rows of 32 threads, twice
static_assert(PT == 512 && SW_TX == 32 && SW_TY == 32, "streamed-pass thread layout");

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// one bounded probe of the phase: the thread sleeps (up to the hint, 20 us)
// until the phase completes instead of spinning on issue slots
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity), "r"(20000u)
      : "memory");
  return done != 0;
}
// wait for the phase of `parity` to complete, giving up after ~2 s of SM clock
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > BAR_WAIT_CYCLES) return false;
  return true;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// orders this thread's (and, through the barriers before it, the grid's)
// generic-proxy view of global memory before its async-proxy (TMA) reads
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// 3D tiled TMA load of one box into shared memory, completing on `bar`.
// The x coordinate must be a multiple of 16 bytes' worth of elements (the
// callers use x0 - 4 for 4-byte data and x0 - 16 for bytes, x0 % 32 == 0).
__device__ __forceinline__ void tma_load3(unsigned dst, const void* map, int x, int y, int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Byte layout of one ring slot: x of two planes [2][by][SW_BX], b likewise,
// the flags [2][by][SW_FBX]; every part a multiple of 128 bytes.
template <class T>
struct SwSlot {
  static constexpr int BY = SW_TY + 2 * SW_HY;
  static constexpr int XB = SW_BX * BY * (int)sizeof(T);  // one plane of x or b
  static constexpr int FB = SW_FBX * BY;                  // one plane of flags
  static constexpr int BYTES = 4 * XB + 2 * FB;
};

// The level's constants for one phase, held in registers for the streamed
// passes (the hierarchy itself sits in shared memory, where every field
// read is a load).
template <class T>
struct SwGrid {
  int n0, n1, n2;
  T wr[6];  // wall weights (xlo, xhi, ylo, yhi, zlo, zhi), as in the level's operator
  T h2e, ceps, lh, idg;
  __device__ SwGrid(const Op<T>& o, int p) {
    n0 = o.n[0];
    n1 = o.n[1];
    n2 = o.n[2];
    for (int q = 0; q < 6; ++q) wr[q] = o.wr[q];
    h2e = o.h2e[p];
    ceps = o.ceps[p];
    lh = o.lh[p];
    idg = o.idg[p];
  }
  // 1 / (dg + lh) for a cell whose stencil gave dg (dg = 6 away from the walls)
  __device__ __forceinline__ T dinv(T dg) const { return dg == T(6) ? idg : rcp_rn(dg + lh); }
};

// Implicit stencil sum and diagonal count of reg_stencil, same terms in the
// same order, at a cell next to a domain wall (box index e, planes Xm, Xc, Xp).
template <class T>
__device__ __noinline__ void sw_wall_stencil(const SwGrid<T>& g, const T* Xm, const T* Xc, const T* Xp, int e, int i,
                                             int j, int k, T& sum_out, T& dg_out) {
  const T third = T(1) / T(3);
  T sum = T(0);
  T dg = T(0);
  if (i > 0) {
    sum += Xc[e - 1];
    dg += T(1);
  } else if (g.wr[0] != T(0)) {
    sum += Xc[e + 1] * (g.wr[0] * third);
    dg += T(3) * g.wr[0];
  }
  if (i < g.n0 - 1) {
    sum += Xc[e + 1];
    dg += T(1);
  } else if (g.wr[1] != T(0)) {
    sum += Xc[e - 1] * (g.wr[1] * third);
    dg += T(3) * g.wr[1];
  }
  if (j > 0) {
    sum += Xc[e - SW_BX];
    dg += T(1);
  } else if (g.wr[2] != T(0)) {
    sum += Xc[e + SW_BX] * (g.wr[2] * third);
    dg += T(3) * g.wr[2];
  }
  if (j < g.n1 - 1) {
    sum += Xc[e + SW_BX];
    dg += T(1);
  } else if (g.wr[3] != T(0)) {
    sum += Xc[e - SW_BX] * (g.wr[3] * third);
    dg += T(3) * g.wr[3];
  }
  if (k > 0) {
    sum += Xm[e];
    dg += T(1);
  } else if (g.wr[4] != T(0)) {
    sum += Xp[e] * (g.wr[4] * third);
    dg += T(3) * g.wr[4];
  }
  if (k < g.n2 - 1) {
    sum += Xp[e];
    dg += T(1);
  } else if (g.wr[5] != T(0)) {
    sum += Xm[e] * (g.wr[5] * third);
    dg += T(3) * g.wr[5];
  }
  sum_out = sum;
  dg_out = dg;
}

// The passes address the ring as one array sm of T (and bytes sb for the
// flags), by 32-bit element indices: a cell is X (its place in its plane's x
// box), M and P (the same place in the planes below and above), Bi (b) and
// Fi (its flag byte); neighbours in x and y are X -+ 1 and X -+ SW_BX.

// The wall stencil of the cell at X, from indices.
template <class T>
__device__ __forceinline__ void sw_wall_at(const SwGrid<T>& g, const T* sm, int X, int M, int P, int i, int j, int k,
                                           T& sum, T& dg) {
  sw_wall_stencil(g, sm + (M - X), sm, sm + (P - X), X, i, j, k, sum, dg);
}

// A thread's two cells of a tile row in the sweep, fixed for an item:
// column A is relaxed as red on planes a = z0 - 1 + 2s and as black on the
// planes between, column B the other way round.  Their indices in a plane
// box (e) and flag box (f), whether each is on the grid (in) and whether its
// x and y neighbours all are (xy).
struct SwCols {
  int iA, iB, eA, eB, fA, fB;
  bool inA, inB, xyA, xyB;
};

// Relaxes the pair's cells (A: indices XA, MA, PA, BA, FA in plane kA; B
// likewise) when each is a regular cell of the phase (flag value pbit) and
// its plane takes part (act).  Both new values are formed before either is
// stored, as two independent chains; the interior formula applies where the
// cell and its plane are away from the walls (fast), the wall stencil
// elsewhere.  The two cells never read each other.
template <class T>
__device__ __forceinline__ void sw_pair(const SwGrid<T>& g, unsigned pbit, T* sm, const unsigned char* sb,
                                        const SwCols& cl, int j, int XA, int MA, int PA, int BA, int FA, bool actA,
                                        bool fastA, int kA, int XB, int MB, int PB, int BB, int FB, bool actB,
                                        bool fastB, int kB) {
  // every index here is inside the ring, whatever the cell
  const T sA = ((((sm[XA - 1] + sm[XA + 1]) + sm[XA - SW_BX]) + sm[XA + SW_BX]) + sm[MA]) + sm[PA];
  const T sB = ((((sm[XB - 1] + sm[XB + 1]) + sm[XB - SW_BX]) + sm[XB + SW_BX]) + sm[MB]) + sm[PB];
  const T vA = (g.h2e * sm[BA] + sA) * g.idg;
  const T vB = (g.h2e * sm[BB] + sB) * g.idg;
  const bool rA = actA && (sb[FA] & 7u) == pbit;
  const bool rB = actB && (sb[FB] & 7u) == pbit;
  if (rA) {
    if (fastA) {
      sm[XA] = vA;
    } else {
      T sum, dg;
      sw_wall_at(g, sm, XA, MA, PA, cl.iA, j, kA, sum, dg);
      sm[XA] = (g.h2e * sm[BA] + sum) * g.dinv(dg);
    }
  }
  if (rB) {
    if (fastB) {
      sm[XB] = vB;
    } else {
      T sum, dg;
      sw_wall_at(g, sm, XB, MB, PB, cl.iB, j, kB, sum, dg);
      sm[XB] = (g.h2e * sm[BB] + sum) * g.dinv(dg);
    }
  }
}

// Relaxes cell (i, j, k) at indices X, M, P, Bi, Fi when it is on the grid
// and a regular cell of the phase (flag value pbit); kin: k is not on a wall
// plane.  Cells off the grid, cut cells and cells of the other phase or
// without an unknown are left alone.
template <class T>
__device__ __forceinline__ void sw_relax_at(const SwGrid<T>& g, unsigned pbit, T* sm, const unsigned char* sb, int X,
                                            int M, int P, int Bi, int Fi, int i, int j, int k, bool kin) {
  if ((unsigned)i >= (unsigned)g.n0 || (unsigned)j >= (unsigned)g.n1) return;
  if ((sb[Fi] & 7u) != pbit) return;  // regular: one phase, no sparse row
  if (kin && (unsigned)(i - 1) < (unsigned)(g.n0 - 2) && (unsigned)(j - 1) < (unsigned)(g.n1 - 2)) {
    const T sum = ((((sm[X - 1] + sm[X + 1]) + sm[X - SW_BX]) + sm[X + SW_BX]) + sm[M]) + sm[P];
    sm[X] = (g.h2e * sm[Bi] + sum) * g.idg;
    return;
  }
  T sum, dg;
  sw_wall_at(g, sm, X, M, P, i, j, k, sum, dg);
  sm[X] = (g.h2e * sm[Bi] + sum) * g.dinv(dg);
}

// Residual b - A x of the regular cell (i, j, k) at indices X, M, P, Bi,
// with the terms and order of cell_residual; fast: the cell is away from
// every wall (the interior formula applies).
template <class T>
__device__ __forceinline__ T sw_resid(const SwGrid<T>& g, const T* sm, int X, int M, int P, int Bi, bool fast, int i,
                                      int j, int k) {
  if (fast) {
    const T sum = ((((sm[X - 1] + sm[X + 1]) + sm[X - SW_BX]) + sm[X + SW_BX]) + sm[M]) + sm[P];
    return sm[Bi] - g.ceps * ((T(6) + g.lh) * sm[X] - sum);
  }
  T sum, dg;
  sw_wall_at(g, sm, X, M, P, i, j, k, sum, dg);
  return sm[Bi] - g.ceps * ((dg + g.lh) * sm[X] - sum);
}

// The work items of a streamed pass over level l: item index r < nitems is
// tile (r % ntx, (r / ntx) % nty) and z-chunk r / (ntx nty) in the gas phase;
// r >= nitems is the item list1[r - nitems] in the dielectric phase.
template <class T>
struct SwItem {
  int x0, y0, z0, z1, p;
  __device__ void at(const SweepLev<T>& sw, int n2, int r) {
    int it = r;
    p = 0;
    if (r >= sw.nitems) {
      it = sw.list1[r - sw.nitems];
      p = 1;
    }
    const int tx = it % sw.ntx, q = it / sw.ntx;
    x0 = tx * SW_TX;
    y0 = (q % sw.nty) * SW_TY;
    z0 = (q / sw.nty) * sw.zc;
    z1 = min(z0 + sw.zc, n2);
  }
};

// The kernel's dynamic shared memory, named here rather than passed in: the
// passes are out-of-line functions, and through a pointer argument the
// compiler could not tell that the ring is shared memory (generic instead of
// shared-window loads and stores in the inner loops).
extern __shared__ __align__(128) unsigned char sw_smem[];

// The shared-memory head: SW_NS mbarriers, then a failure flag; the ring
// starts at SW_HEAD, on a 128-byte boundary (the host adds 128 bytes of slack).
__device__ __forceinline__ unsigned char* sw_ring(unsigned char* dyn) {
  return dyn + SW_HEAD + ((128u - (smem_u32(dyn + SW_HEAD) & 127u)) & 127u);
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Issues the two-plane copies of a streamed pass in order (thread 0 only).
// The items come from the level's ticket counter, so that CTAs which drew
// cheap items (inside an electrode, no unknowns) take more of them: a ticket
// below the pass's item count is the next item, whose index goes into the
// shared queue (entry nk % SW_QN) before its first copy is issued; its copies
// then start at plane z0 - lead, two planes each.  A ticket past the end puts
// -1 in the queue and, in place of a copy, a plain arrival on the next
// slot's mbarrier.  The queue entry is published by that copy's (or
// arrival's) completion: the arrival releases it and the waiting threads
// acquire it.
template <class T>
struct SwIssue {
  static constexpr int LEAD = 2;  // copies start two planes before the item
  int ig, iq, ng, nk, state;      // state 0: an item's copies to issue, 1: the end to mark, 2: done
  SwItem<T> it;
  __device__ void start(const SweepLev<T>& sw, int n2, int* ctr) {
    ig = 0;
    iq = 0;
    nk = 0;
    grab(sw, n2, ctr);
  }
  __device__ void grab(const SweepLev<T>& sw, int n2, int* ctr) {
    volatile int* q = (volatile int*)(sw_smem + SW_QOFF);
    const int t = atomicAdd(ctr, 1);
    if (t < sw.nitems + sw.n1items) {
      it.at(sw, n2, t);
      ng = (it.z1 - it.z0 + 2 * LEAD) >> 1;
      state = 0;
      q[nk % SW_QN] = t;
    } else {
      state = 1;
      q[nk % SW_QN] = -1;
    }
    ++nk;
  }
  __device__ void run(const SweepLev<T>& sw, int n2, int* ctr, unsigned char* ring, unsigned bar0, int limit) {
    using L = SwSlot<T>;
    const unsigned char* maps = (const unsigned char*)sw.maps;
    while (iq < limit && state != 2) {
      const int s = iq % SW_NS;
      const unsigned bar = bar0 + 8 * s;
      ++iq;
      if (state == 1) {
        mbar_arrive(bar);
        state = 2;
        break;
      }
      const unsigned base = smem_u32(ring + s * L::BYTES);
      const int z = it.z0 - LEAD + 2 * ig;
      mbar_expect_tx(bar, (unsigned)L::BYTES);
      tma_load3(base, maps + 128 * (2 * sw.par + it.p), it.x0 - SW_HX, it.y0 - SW_HY, z, bar);
      tma_load3(base + 2 * L::XB, maps + 128 * (4 + it.p), it.x0 - SW_HX, it.y0 - SW_HY, z, bar);
      tma_load3(base + 4 * L::XB, maps + 128 * 6, it.x0 - SW_FHX, it.y0 - SW_HY, z, bar);
      if (++ig == ng) {
        ig = 0;
        grab(sw, n2, ctr);
      }
    }
  }
};

// After a completed pass (thread 0 of each worker CTA): the last CTA done
// resets the pass's ticket counter and done count for the next pass, which
// starts after a grid barrier.  Every CTA counts itself only after the
// ticket that ended its pass came back.
__device__ __forceinline__ void sw_pass_done(int* ctr, int workers) {
  __threadfence();
  if (atomicAdd(ctr + 1, 1) == workers - 1) {
    atomicExch(ctr, 0);
    atomicExch(ctr + 1, 0);
  }
}

// Waits (bounded) until loads up to index `need` have landed; false on expiry.
__device__ __forceinline__ bool sw_wait_upto(unsigned bar0, int& waited, int need) {
  for (; waited <= need; ++waited)
    if (!mbar_wait(bar0 + 8 * (waited % SW_NS), (unsigned)((waited / SW_NS) & 1))) return false;
  return true;
}

// After a failure: raise the grid's error word and let this CTA's copies in
// flight land (bounded), so that none writes into shared memory after return.
__device__ __forceinline__ void sw_drain(const Ctx& c, unsigned bar0, int waited, int issued) {
  if (threadIdx.x == 0) {
    if (c.B.err) atomicOr(c.B.err, 1);
    for (; waited < issued; ++waited)
      if (!mbar_wait(bar0 + 8 * (waited % SW_NS), (unsigned)((waited / SW_NS) & 1))) break;
  }
}

// One fused pass over the regular cells of grid level l (SweepLev on),
// x -> alt, then x and alt swap in this CTA's copy of the hierarchy.  CTA 0
// of the group keeps the coarse levels in its shared memory and sits the
// pass out; the other CTAs draw the items from the level's ticket counter.
//
// Item with planes [z0, z1): copy g holds planes z0 - 2 + 2g and the next;
// step s (s = 0 .. Z/2 + 1, Z = z1 - z0) relaxes red on planes a, a + 1
// (a = z0 - 1 + 2s; within [z0 - 1, z1], the ring plane at each end
// included), block barrier, black on planes a - 1, a (within [z0, z1)),
// stores planes a - 3, a - 2 (within [z0, z1)), then refills the slots of
// the copies below g = s - 1, which no later step reads.
template <class T>
__device__ __noinline__ bool ph_sweep3d(const Hier<T>& Hc, int l, const Ctx& c) {
  unsigned char* const dyn = sw_smem;
  using L = SwSlot<T>;
  Hier<T>& H = const_cast<Hier<T>&>(Hc);
  Op<T>& o = H.op[l];
  SweepLev<T>& sw = H.sw[l];
  const int nw = c.gsize - 1;
  const int n2 = o.n[2];
  unsigned long long* bars = (unsigned long long*)dyn;
  volatile int* sfail = (volatile int*)(dyn + 8 * SW_NS);
  volatile int* sq = (volatile int*)(dyn + SW_QOFF);
  unsigned char* ring = sw_ring(dyn);
  const unsigned bar0 = smem_u32(bars);
  // the ring by element indices: slot g starts at re + g SE, its second
  // plane's x box XE further; its flag boxes at byte FO of the slot
  T* const sm = (T*)dyn;
  const unsigned char* const sb = dyn;
  constexpr int SE = L::BYTES / (int)sizeof(T), XE = L::XB / (int)sizeof(T), FO = 4 * L::XB;
  const int re = (int)(ring - dyn) / (int)sizeof(T);
  bool ok = true;
  if (c.gcta > 0) {
    if (threadIdx.x == 0) {
      for (int s = 0; s < SW_NS; ++s) mbar_init(bar0 + 8 * s, 1);
      fence_mbar_init();
      *sfail = 0;
    }
    __syncthreads();
    SwIssue<T> iss;
    if (threadIdx.x == 0) {
      fence_async_global();  // x was last written by generic stores of other CTAs
      iss.start(sw, n2, sw.tick);
      iss.run(sw, n2, sw.tick, ring, bar0, SW_NS);
    }
    // thread mapping: the tile's cells of one colour, 16 per row; the ring's
    // red cells of two planes (2 x (2 rows of 17 + 32 row ends)) by the last
    // 132 threads, away from warp 0, which issues the copies
    const int t = threadIdx.x;
    const int tr = t >> 4, tm = t & 15;
    const int tring = (int)blockDim.x - 1 - t;
    const int ly_in = SW_HY + tr;                         // this thread's tile row in the boxes
    const int e_in = ly_in * SW_BX + SW_HX + 2 * tm;      // its even-parity cell of the row
    const int f_in = ly_in * SW_FBX + SW_FHX + 2 * tm;    // the same in the flag box
    // the ring cell of this thread, if any: box position without the colour offset
    int rq_ly = 0, rq_lx = 0, rq_h = -1;
    {
      const int tq = tring < 66 ? tring : tring - 66;
      if (tring < 132) {
        rq_h = tring < 66 ? 0 : 1;
        if (tq < 34) {  // ring rows above and below the tile, 17 red cells each
          rq_ly = tq < 17 ? SW_HY - 1 : SW_HY + SW_TY;
          rq_lx = SW_HX - 1 + 2 * (tq < 17 ? tq : tq - 17);  // lx = rq_lx + ((j + r + 1) & 1)
        } else {       // the ring cell at the left or right end of a tile row
          rq_ly = SW_HY + tq - 34;
          rq_lx = -1;  // lx = 3 or 36 by the colour
        }
      }
    }
    int qb = 0, waited = 0;
    for (int k = 0;; ++k) {
      // the item's first copy, or the end of the pass, completes at index qb
      if (!sw_wait_upto(bar0, waited, qb)) *sfail = 1;
      __syncthreads();
      if (*sfail) {
        ok = false;
        break;
      }
      const int r = sq[k % SW_QN];
      if (r < 0) break;
      SwItem<T> it;
      it.at(sw, n2, r);
      const SwGrid<T> g(o, it.p);
      const unsigned pbit = 1u << it.p;
      T* const alt = sw.alt[it.p];
      const int x0 = it.x0, y0 = it.y0, z0 = it.z0, z1 = it.z1;
      const int G = (z1 - z0 + 4) >> 1, S = ((z1 - z0) >> 1) + 2;
      const int j_in = y0 + tr;
      const int rq_j = y0 - SW_HY + rq_ly;
      // this thread's pair of cells, fixed for the item: column A is red in
      // planes of the parity of z0 - 1
      SwCols cl;
      {
        const int oA = (j_in + z0 + 1) & 1, oB = oA ^ 1;
        cl.iA = x0 + 2 * tm + oA;
        cl.iB = x0 + 2 * tm + oB;
        cl.eA = e_in + oA;
        cl.eB = e_in + oB;
        cl.fA = f_in + oA;
        cl.fB = f_in + oB;
        const bool jin = j_in < g.n1, jxy = (unsigned)(j_in - 1) < (unsigned)(g.n1 - 2);
        cl.inA = jin && cl.iA < g.n0;
        cl.inB = jin && cl.iB < g.n0;
        cl.xyA = jxy && (unsigned)(cl.iA - 1) < (unsigned)(g.n0 - 2);
        cl.xyB = jxy && (unsigned)(cl.iB - 1) < (unsigned)(g.n0 - 2);
      }
      // stores: this thread's column rx of tile rows ry0 and ry0 + 16 (the
      // kernel runs 512 threads: 16 rows of 32 per pass over the tile)
      const int rx = t & 31, ry0 = t >> 5;
      const bool sx = x0 + rx < g.n0;
      const bool st0 = sx && y0 + ry0 < g.n1, st1 = sx && y0 + ry0 + 16 < g.n1;
      T* const dst0 = alt + ((long long)z0 * g.n1 + y0 + ry0) * g.n0 + x0 + rx;
      const long long plane = (long long)g.n0 * g.n1, row16 = 16LL * g.n0;
      const int sb0 = (SW_HY + ry0) * SW_BX + SW_HX + rx, sb1 = sb0 + 16 * SW_BX;
      // copy g of this item sits in slot (qb + g) % SW_NS; the element
      // indices of the slots of copies s - 1, s, s + 1 rotate by one per step
      int E0 = re + ((qb + SW_NS - 1) % SW_NS) * SE, E1 = re + (qb % SW_NS) * SE, E2 = re + ((qb + 1) % SW_NS) * SE;
      for (int s = 0; s < S; ++s) {
        if (!sw_wait_upto(bar0, waited, qb + min(s + 1, G - 1))) *sfail = 1;
        const int a = z0 - 1 + 2 * s;
        // planes a - 3, a - 2 in copy s - 1 (slot E0); a - 1, a in copy s
        // (E1); a + 1, a + 2 in copy s + 1 (E2); in a slot the x boxes of
        // its two planes, then their b boxes, then their flag boxes
        const int F1 = E1 * (int)sizeof(T) + FO, F2 = E2 * (int)sizeof(T) + FO;
        // whether planes a - 1, a, a + 1 lie off the z walls
        const bool km = a - 1 > 0 && a - 1 < n2 - 1, k0 = a > 0 && a < n2 - 1, kp = a + 1 > 0 && a + 1 < n2 - 1;
        // red: A in plane a (copy s, second plane), B in plane a + 1 (copy
        // s + 1, first): the item's planes and the ring plane at each end
        {
          const int xa = E1 + XE + cl.eA, xb = E2 + cl.eB;
          sw_pair(g, pbit, sm, sb, cl, j_in, xa, xa - XE, E2 + cl.eA, xa + 2 * XE, F1 + L::FB + cl.fA,
                  cl.inA && a >= 0 && a <= z1 && a < n2, cl.xyA && k0, a, xb, E1 + XE + cl.eB, xb + XE,
                  xb + 2 * XE, F2 + cl.fB, cl.inB && a + 1 <= z1 && a + 1 < n2, cl.xyB && kp, a + 1);
        }
        if (rq_h >= 0) {
          const int r = a + rq_h;
          if (r <= z1 && r >= 0 && r < n2) {
            const int lx = rq_lx >= 0 ? rq_lx + ((rq_j + r + 1) & 1) : (((rq_j + r) & 1) ? SW_HX - 1 : SW_HX + SW_TX);
            const int e = rq_ly * SW_BX + lx, f = rq_ly * SW_FBX + lx + (SW_FHX - SW_HX);
            if (rq_h == 0) {
              const int x = E1 + XE + e;
              sw_relax_at(g, pbit, sm, sb, x, x - XE, E2 + e, x + 2 * XE, F1 + L::FB + f, x0 - SW_HX + lx, rq_j, r,
                          k0);
            } else {
              const int x = E2 + e;
              sw_relax_at(g, pbit, sm, sb, x, E1 + XE + e, x + XE, x + 2 * XE, F2 + f, x0 - SW_HX + lx, rq_j, r,
                          kp);
            }
          }
        }
        fence_async_smem();
        __syncthreads();
        if (*sfail) {
          ok = false;
          break;
        }
        // black: A in plane a - 1 (copy s, first plane), B in plane a (copy
        // s, second): the item's planes only
        {
          const int xa = E1 + cl.eA, xb = E1 + XE + cl.eB;
          sw_pair(g, pbit, sm, sb, cl, j_in, xa, E0 + XE + cl.eA, xa + XE, xa + 2 * XE, F1 + cl.fA,
                  cl.inA && a - 1 >= z0 && a - 1 < z1, cl.xyA && km, a - 1, xb, xb - XE, E2 + cl.eB, xb + 2 * XE,
                  F1 + L::FB + cl.fB, cl.inB && a >= z0 && a < z1, cl.xyB && k0, a);
        }
        // store planes a - 3, a - 2 (copy s - 1; final since the last step):
        // the tile's cells as they stand in the box, the phase's regular
        // cells relaxed, the rest as loaded (cut cells as given; cells
        // without an unknown of the phase are never read through this array)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = a - 3 + h;
          if (q < z0 || q >= z1) continue;
          const int X = E0 + h * XE;
          T* const d = dst0 + (q - z0) * plane;
          if (st0) d[0] = sm[X + sb0];
          if (st1) d[row16] = sm[X + sb1];
        }
        // copies below s - 1 are read by no later step: refill their slots
        if (t == 0) iss.run(sw, n2, sw.tick, ring, bar0, qb + max(0, s - 1) + SW_NS);
        E0 = E1;
        E1 = E2;
        E2 = E2 + SE == re + SW_NS * SE ? re : E2 + SE;
      }
      if (!ok) break;
      qb += G;
    }
    if (!ok) sw_drain(c, bar0, waited, t == 0 ? iss.iq : 0);
    else if (t == 0) sw_pass_done(sw.tick, nw);
    __syncthreads();
    if (t == 0)
      for (int s = 0; s < SW_NS; ++s) mbar_inval(bar0 + 8 * s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // the new iterate is in alt: swap the buffers of this CTA's view
    for (int p = 0; p < 2; ++p) {
      T* tmp = o.x[p];
      o.x[p] = sw.alt[p];
      sw.alt[p] = tmp;
    }
    sw.par ^= 1;
  }
  return ok;
}

// Residual + restriction of grid level l (SweepLev on) onto level l + 1
// (half the cells per axis): coarse b = mean of the children's residuals
// (cut children from the sparse residual rows in tmp), coarse x = 0, per
// phase.  The level streams through the same ring: copy g holds planes
// z0 - 2 + 2g and the next; step s forms the residuals of planes z0 + 2s and
// z0 + 2s + 1, which are the children of one coarse plane: pairs of x
// neighbours combine by a shuffle, the coarse plane is stored, and after the
// step's block barrier the slots of the copies below g = s + 1 are refilled.
template <class T>
__device__ __noinline__ bool ph_restrict3d(const Hier<T>& Hc, int l, const Ctx& c) {
  unsigned char* const dyn = sw_smem;
  using L = SwSlot<T>;
  const Hier<T>& H = Hc;
  const Op<T>& o = H.op[l];
  const Op<T>& co = H.op[l + 1];
  const SweepLev<T>& sw = H.sw[l];
  const int nw = c.gsize - 1;
  const int n2 = o.n[2];
  unsigned long long* bars = (unsigned long long*)dyn;
  volatile int* sfail = (volatile int*)(dyn + 8 * SW_NS);
  volatile int* sq = (volatile int*)(dyn + SW_QOFF);
  unsigned char* ring = sw_ring(dyn);
  const unsigned bar0 = smem_u32(bars);
  const T* const sm = (const T*)dyn;  // the ring by element indices, as in the sweep
  const unsigned char* const sb = dyn;
  constexpr int SE = L::BYTES / (int)sizeof(T), XE = L::XB / (int)sizeof(T), FO = 4 * L::XB;
  const int re = (int)(ring - dyn) / (int)sizeof(T);
  bool ok = true;
  if (c.gcta > 0) {
    if (threadIdx.x == 0) {
      for (int s = 0; s < SW_NS; ++s) mbar_init(bar0 + 8 * s, 1);
      fence_mbar_init();
      *sfail = 0;
    }
    __syncthreads();
    SwIssue<T> iss;
    if (threadIdx.x == 0) {
      fence_async_global();
      iss.start(sw, n2, sw.tick + 2);
      iss.run(sw, n2, sw.tick + 2, ring, bar0, SW_NS);
    }
    // thread t: fine cells (2 cx + h, 2 cy + v), v = 0, 1, of coarse cell
    // (cx, cy) = ((t >> 1) & 15, t >> 5) in both planes of a step
    const int t = threadIdx.x;
    const int hx = t & 1, ccx = (t >> 1) & 15, ccy = t >> 5;
    const int rx = 2 * ccx + hx, lx = SW_HX + rx;
    const int e0 = (SW_HY + 2 * ccy) * SW_BX + lx;                    // row 2 cy in the x / b boxes
    const int f0 = (SW_HY + 2 * ccy) * SW_FBX + lx + (SW_FHX - SW_HX);  // and in the flag box
    const T scale = T(1) / T(8);
    const int cn0 = co.n[0], cn1 = co.n[1];
    int qb = 0, waited = 0;
    for (int k = 0;; ++k) {
      // the item's first copy, or the end of the pass, completes at index qb
      if (!sw_wait_upto(bar0, waited, qb)) *sfail = 1;
      __syncthreads();
      if (*sfail) {
        ok = false;
        break;
      }
      const int r = sq[k % SW_QN];
      if (r < 0) break;
      SwItem<T> it;
      it.at(sw, n2, r);
      const SwGrid<T> g(o, it.p);
      const int p = it.p;
      const unsigned pbit = 1u << p;
      const int x0 = it.x0, y0 = it.y0, z0 = it.z0, z1 = it.z1;
      const int G = (z1 - z0 + 4) >> 1, S = (z1 - z0) >> 1;
      T* const cb = co.b[p];
      T* const cx = co.x[p];
      // this thread's fine cells (i, j0 + v), fixed for the item, and its
      // coarse cell (the even-x thread of each pair stores it)
      const int i = x0 + rx, j0 = y0 + 2 * ccy;
      const bool iin = i < g.n0, ixy = (unsigned)(i - 1) < (unsigned)(g.n0 - 2);
      const bool in0 = iin && j0 < g.n1, in1 = iin && j0 + 1 < g.n1;
      const bool xy0 = ixy && (unsigned)(j0 - 1) < (unsigned)(g.n1 - 2);
      const bool xy1 = ixy && (unsigned)j0 < (unsigned)(g.n1 - 2);
      const int ci = (x0 >> 1) + ccx, cj = (y0 >> 1) + ccy;
      const bool cown = hx == 0 && ci < cn0 && cj < cn1 && cb;
      const long long cplane = (long long)cn0 * cn1;
      const long long Cz0 = ((long long)(z0 >> 1) * cn1 + cj) * cn0 + ci;
      // copies s, s + 1, s + 2 hold planes z0 + 2s - 2 .. z0 + 2s + 3; the
      // element indices of their slots rotate by one per step
      int E0 = re + (qb % SW_NS) * SE, E1 = re + ((qb + 1) % SW_NS) * SE, E2 = re + ((qb + 2) % SW_NS) * SE;
      for (int s = 0; s < S; ++s) {
        if (!sw_wait_upto(bar0, waited, qb + min(s + 2, G - 1))) *sfail = 1;
        // the coarse cell's flags, requested before the residuals so that the
        // load overlaps them
        const long long C = Cz0 + s * cplane;
        const unsigned cfl = cown ? co.flags[C] : 0u;
        const int F1 = E1 * (int)sizeof(T) + FO;
        T acc = T(0);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          // plane z0 + 2s (copy s + 1, first) then z0 + 2s + 1 (copy s + 1,
          // second); the planes below and above in copies s, s + 1, s + 2
          const int z = z0 + 2 * s + h;
          const int X = E1 + h * XE + e0;
          const int M = (h == 0 ? E0 + XE : E1) + e0, P = (h == 0 ? E1 + XE : E2) + e0;
          const bool kin = z > 0 && z < n2 - 1;
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int j = j0 + v;
            if (!(v == 0 ? in0 : in1)) continue;
            const unsigned f = sb[F1 + h * L::FB + f0 + v * SW_FBX];
            if (!(f & pbit)) continue;
            if (f & F_IRR) {
              const long long cc = ((long long)z * g.n1 + j) * g.n0 + i;
              acc += o.tmp[2 * (long long)o.irr_of_cell[cc] + p];
              continue;
            }
            const int dv = v * SW_BX;
            acc += sw_resid(g, sm, X + dv, M + dv, P + dv, X + dv + 2 * XE, kin && (v == 0 ? xy0 : xy1), i, j, z);
          }
        }
        // the pair of x neighbours of one coarse cell sits in lanes t, t ^ 1
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (cown) {
          cb[C] = ((cfl >> p) & 1u) ? acc * scale : T(0);
          cx[C] = T(0);
        }
        __syncthreads();
        if (*sfail) {
          ok = false;
          break;
        }
        // copies below s + 1 (all of the item's after its last step) are read
        // by no later step: refill their slots
        if (t == 0) iss.run(sw, n2, sw.tick + 2, ring, bar0, qb + (s == S - 1 ? G : s + 1) + SW_NS);
        E0 = E1;
        E1 = E2;
        E2 = E2 + SE == re + SW_NS * SE ? re : E2 + SE;
      }
      if (!ok) break;
      qb += G;
    }
    if (!ok) sw_drain(c, bar0, waited, t == 0 ? iss.iq : 0);
    else if (t == 0) sw_pass_done(sw.tick + 2, nw);
    __syncthreads();
    if (t == 0)
      for (int s = 0; s < SW_NS; ++s) mbar_inval(bar0 + 8 * s);
  }
  __syncthreads();
  return ok;
}

}  // namespace ebp
