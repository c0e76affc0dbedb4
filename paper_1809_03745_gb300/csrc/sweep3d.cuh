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
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
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
  unsigned bcm;  // bit s set: Dirichlet wall on side s (xlo, xhi, ylo, yhi, zlo, zhi)
  T h2e, ceps;
  __device__ SwGrid(const Op<T>& o, int p) {
    n0 = o.n[0];
    n1 = o.n[1];
    n2 = o.n[2];
    bcm = 0u;
    for (int q = 0; q < 6; ++q) bcm |= (o.bc[q] ? 1u : 0u) << q;
    h2e = o.h2e[p];
    ceps = o.ceps[p];
  }
};

// Implicit stencil sum and diagonal count of reg_stencil, same terms in the
// same order, at a cell next to a domain wall (box index e, planes Xm, Xc, Xp).
template <class T>
__device__ __noinline__ void sw_wall_stencil(const SwGrid<T>& g, const T* Xm, const T* Xc, const T* Xp, int e, int i,
                                             int j, int k, T& sum_out, int& dg_out) {
  const T third = T(1) / T(3);
  T sum = T(0);
  int dg = 0;
  if (i > 0) {
    sum += Xc[e - 1];
    dg += 1;
  } else if (g.bcm & 1u) {
    sum += Xc[e + 1] * third;
    dg += 3;
  }
  if (i < g.n0 - 1) {
    sum += Xc[e + 1];
    dg += 1;
  } else if (g.bcm & 2u) {
    sum += Xc[e - 1] * third;
    dg += 3;
  }
  if (j > 0) {
    sum += Xc[e - SW_BX];
    dg += 1;
  } else if (g.bcm & 4u) {
    sum += Xc[e + SW_BX] * third;
    dg += 3;
  }
  if (j < g.n1 - 1) {
    sum += Xc[e + SW_BX];
    dg += 1;
  } else if (g.bcm & 8u) {
    sum += Xc[e - SW_BX] * third;
    dg += 3;
  }
  if (k > 0) {
    sum += Xm[e];
    dg += 1;
  } else if (g.bcm & 16u) {
    sum += Xp[e] * third;
    dg += 3;
  }
  if (k < g.n2 - 1) {
    sum += Xp[e];
    dg += 1;
  } else if (g.bcm & 32u) {
    sum += Xm[e] * third;
    dg += 3;
  }
  sum_out = sum;
  dg_out = dg;
}

// Relaxes cell (i, j, k), at index e of the x / b boxes and ef of the flag
// box, of planes Xc (k), Xm, Xp with right-hand side B and flags F when it
// is a regular cell of phase p (flag value pbit = 1 << p); kin: k is not on
// a wall plane.  Cells off the grid, cut cells and cells of the other phase
// or without an unknown are left alone.
template <class T>
__device__ __forceinline__ void sw_relax_at(const SwGrid<T>& g, T* Xc, const T* Xm, const T* Xp, const T* B,
                                            const unsigned char* F, unsigned pbit, int i, int j, int k, bool kin,
                                            int e, int ef) {
  if ((unsigned)i >= (unsigned)g.n0 || (unsigned)j >= (unsigned)g.n1) return;
  if ((F[ef] & 7u) != pbit) return;  // regular: one phase, no sparse row
  if (kin && (unsigned)(i - 1) < (unsigned)(g.n0 - 2) && (unsigned)(j - 1) < (unsigned)(g.n1 - 2)) {
    const T sum = ((((Xc[e - 1] + Xc[e + 1]) + Xc[e - SW_BX]) + Xc[e + SW_BX]) + Xm[e]) + Xp[e];
    Xc[e] = (g.h2e * B[e] + sum) * inv_count(6, T(0));
    return;
  }
  T sum;
  int dg;
  sw_wall_stencil(g, Xm, Xc, Xp, e, i, j, k, sum, dg);
  Xc[e] = (g.h2e * B[e] + sum) * inv_count(dg, T(0));
}

// Residual b - A x of the regular cell (i, j, k) at box position (lx, ly),
// with the terms and order of cell_residual.
template <class T>
__device__ __forceinline__ T sw_resid(const SwGrid<T>& g, const T* Xc, const T* Xm, const T* Xp, const T* B, int i,
                                      int j, int k, bool kin, int lx, int ly) {
  const int e = ly * SW_BX + lx;
  if (kin && (unsigned)(i - 1) < (unsigned)(g.n0 - 2) && (unsigned)(j - 1) < (unsigned)(g.n1 - 2)) {
    const T sum = ((((Xc[e - 1] + Xc[e + 1]) + Xc[e - SW_BX]) + Xc[e + SW_BX]) + Xm[e]) + Xp[e];
    return B[e] - g.ceps * ((T)6 * Xc[e] - sum);
  }
  T sum;
  int dg;
  sw_wall_stencil(g, Xm, Xc, Xp, e, i, j, k, sum, dg);
  return B[e] - g.ceps * ((T)dg * Xc[e] - sum);
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

// The shared-memory head: SW_NS mbarriers, then a failure flag; the ring
// starts at SW_HEAD, on a 128-byte boundary (the host adds 128 bytes of slack).
__device__ __forceinline__ unsigned char* sw_ring(unsigned char* dyn) {
  return dyn + SW_HEAD + ((128u - (smem_u32(dyn + SW_HEAD) & 127u)) & 127u);
}

// Issues the two-plane copies of a streamed pass in order (thread 0 only):
// loads iq < limit, item by item, `groups(item)` copies each starting at
// plane z0 - 2.  The cursor (item ik, copy ig within it) advances without
// divisions; an item's geometry is computed when the cursor reaches it.
template <class T>
struct SwIssue {
  int ik, ig, iq, K, ng;
  SwItem<T> it;
  const void *mx, *mb, *mf;
  __device__ void start(const SweepLev<T>& sw, int n2, int w, int nw, int k_total, const unsigned char* maps,
                        int lead) {
    ik = 0;
    ig = 0;
    iq = 0;
    K = k_total;
    if (K > 0) load_item(sw, n2, w, nw, maps, lead);
  }
  __device__ void load_item(const SweepLev<T>& sw, int n2, int w, int nw, const unsigned char* maps, int lead) {
    it.at(sw, n2, w + ik * nw);
    ng = (it.z1 - it.z0 + 2 * lead) >> 1;
    mx = maps + 128 * (2 * sw.par + it.p);
    mb = maps + 128 * (4 + it.p);
    mf = maps + 128 * 6;
  }
  __device__ void run(const SweepLev<T>& sw, int n2, int w, int nw, const unsigned char* maps, unsigned char* ring,
                      unsigned bar0, int limit, int lead) {
    using L = SwSlot<T>;
    while (iq < limit && ik < K) {
      const int s = iq % SW_NS;
      const unsigned bar = bar0 + 8 * s;
      const unsigned base = smem_u32(ring + s * L::BYTES);
      const int z = it.z0 - lead + 2 * ig;
      mbar_expect_tx(bar, (unsigned)L::BYTES);
      tma_load3(base, mx, it.x0 - SW_HX, it.y0 - SW_HY, z, bar);
      tma_load3(base + 2 * L::XB, mb, it.x0 - SW_HX, it.y0 - SW_HY, z, bar);
      tma_load3(base + 4 * L::XB, mf, it.x0 - SW_FHX, it.y0 - SW_HY, z, bar);
      ++iq;
      if (++ig == ng) {
        ig = 0;
        if (++ik < K) load_item(sw, n2, w, nw, maps, lead);
      }
    }
  }
};

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
// pass out; the other CTAs take the items round-robin.
//
// Item with planes [z0, z1): copy g holds planes z0 - 2 + 2g and the next;
// step s (s = 0 .. Z/2 + 1, Z = z1 - z0) relaxes red on planes a, a + 1
// (a = z0 - 1 + 2s; within [z0 - 1, z1], the ring plane at each end
// included), block barrier, black on planes a - 1, a (within [z0, z1)),
// stores planes a - 3, a - 2 (within [z0, z1)), then refills the slots of
// the copies below g = s - 1, which no later step reads.
template <class T>
__device__ __noinline__ bool ph_sweep3d(const Hier<T>& Hc, int l, const Ctx& c, unsigned char* dyn) {
  using L = SwSlot<T>;
  Hier<T>& H = const_cast<Hier<T>&>(Hc);
  Op<T>& o = H.op[l];
  SweepLev<T>& sw = H.sw[l];
  const int nw = c.gsize - 1, w = c.gcta - 1;
  const int n2 = o.n[2];
  const int ntot = sw.nitems + sw.n1items;
  const int K = (w >= 0 && ntot > w) ? (ntot - 1 - w) / nw + 1 : 0;
  unsigned long long* bars = (unsigned long long*)dyn;
  volatile int* sfail = (volatile int*)(dyn + 8 * SW_NS);
  unsigned char* ring = sw_ring(dyn);
  const unsigned bar0 = smem_u32(bars);
  bool ok = true;
  if (K > 0) {
    if (threadIdx.x == 0) {
      for (int s = 0; s < SW_NS; ++s) mbar_init(bar0 + 8 * s, 1);
      fence_mbar_init();
      *sfail = 0;
    }
    __syncthreads();
    const unsigned char* maps = (const unsigned char*)sw.maps;
    SwIssue<T> iss;
    if (threadIdx.x == 0) {
      iss.start(sw, n2, w, nw, K, maps, 2);
      fence_async_global();  // x was last written by generic stores of other CTAs
      iss.run(sw, n2, w, nw, maps, ring, bar0, SW_NS, 2);
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
    for (int k = 0; k < K && ok; ++k) {
      SwItem<T> it;
      it.at(sw, n2, w + k * nw);
      const SwGrid<T> g(o, it.p);
      const unsigned pbit = 1u << it.p;
      T* const alt = sw.alt[it.p];
      const int x0 = it.x0, y0 = it.y0, z0 = it.z0, z1 = it.z1;
      const int G = (z1 - z0 + 4) >> 1, S = ((z1 - z0) >> 1) + 2;
      const int j_in = y0 + tr;
      const int i_even = x0 + 2 * tm;  // the cell at e_in
      const int rq_j = y0 - SW_HY + rq_ly;
      // copy g of this item sits in slot (qb + g) % SW_NS; slot pointers of
      // copies s - 1, s, s + 1 rotate by one per step
      int sl0 = (qb + SW_NS - 1) % SW_NS, sl1 = qb % SW_NS, sl2 = (qb + 1) % SW_NS;
      for (int s = 0; s < S; ++s) {
        if (!sw_wait_upto(bar0, waited, qb + min(s + 1, G - 1))) *sfail = 1;
        const int a = z0 - 1 + 2 * s;
        // planes a - 3, a - 2 in copy s - 1; a - 1, a in copy s; a + 1, a + 2 in copy s + 1
        unsigned char* const C0 = ring + sl0 * L::BYTES;
        unsigned char* const C1 = ring + sl1 * L::BYTES;
        unsigned char* const C2 = ring + sl2 * L::BYTES;
        // red cells of planes a (copy s, second plane) and a + 1 (copy s + 1, first)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = a + h;
          if (r > z1 || r < 0 || r >= n2) continue;
          unsigned char* const Pc = h == 0 ? C1 + L::XB : C2;
          const unsigned char* const Pm = h == 0 ? C1 : C1 + L::XB;
          const unsigned char* const Pp = h == 0 ? C2 : C2 + L::XB;
          const unsigned char* const F = h == 0 ? C1 + 4 * L::XB + L::FB : C2 + 4 * L::XB;
          T* Xc = (T*)Pc;
          const T *Xm = (const T*)Pm, *Xp = (const T*)Pp, *B = (const T*)(Pc + 2 * L::XB);
          const bool kin = r > 0 && r < n2 - 1;
          {
            const int o1 = (j_in + r) & 1;
            sw_relax_at(g, Xc, Xm, Xp, B, F, pbit, i_even + o1, j_in, r, kin, e_in + o1, f_in + o1);
          }
          if (rq_h == h) {
            const int lx = rq_lx >= 0 ? rq_lx + ((rq_j + r + 1) & 1) : (((rq_j + r) & 1) ? SW_HX - 1 : SW_HX + SW_TX);
            sw_relax_at(g, Xc, Xm, Xp, B, F, pbit, x0 - SW_HX + lx, rq_j, r, kin, rq_ly * SW_BX + lx,
                        rq_ly * SW_FBX + lx + (SW_FHX - SW_HX));
          }
        }
        fence_async_smem();
        __syncthreads();
        if (*sfail) {
          ok = false;
          break;
        }
        // black cells of planes a - 1 (copy s, first plane) and a (copy s, second)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = a - 1 + h;
          if (q < z0 || q >= z1) continue;
          unsigned char* const Pc = h == 0 ? C1 : C1 + L::XB;
          const unsigned char* const Pm = h == 0 ? C0 + L::XB : C1;
          const unsigned char* const Pp = h == 0 ? C1 + L::XB : C2;
          const unsigned char* const F = C1 + 4 * L::XB + h * L::FB;
          const int o1 = (j_in + q + 1) & 1;
          sw_relax_at(g, (T*)Pc, (const T*)Pm, (const T*)Pp, (const T*)(Pc + 2 * L::XB), F, pbit, i_even + o1, j_in,
                      q, q > 0 && q < n2 - 1, e_in + o1, f_in + o1);
        }
        // store planes a - 3, a - 2 (copy s - 1; final since the last step):
        // the tile's unknowns of this phase, both colours, cut cells as given
        {
          const int rx = t & 31, i = x0 + rx;
          if (i < g.n0)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int q = a - 3 + h;
              if (q < z0 || q >= z1) continue;
              const T* X = (const T*)(C0 + h * L::XB);
              const unsigned char* F = C0 + 4 * L::XB + h * L::FB;
              T* dst = alt + ((long long)q * g.n1 + y0) * g.n0 + i;
              for (int ry = t >> 5; ry < SW_TY; ry += (int)(blockDim.x >> 5)) {
                if (y0 + ry >= g.n1) break;
                const int ly = SW_HY + ry;
                if (F[ly * SW_FBX + SW_FHX + rx] & pbit) dst[(long long)ry * g.n0] = X[ly * SW_BX + SW_HX + rx];
              }
            }
        }
        // copies below s - 1 are read by no later step: refill their slots
        if (t == 0) iss.run(sw, n2, w, nw, maps, ring, bar0, qb + max(0, s - 1) + SW_NS, 2);
        sl0 = sl1;
        sl1 = sl2;
        sl2 = sl2 + 1 == SW_NS ? 0 : sl2 + 1;
      }
      qb += G;
    }
    if (!ok) sw_drain(c, bar0, waited, t == 0 ? iss.iq : 0);
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
__device__ __noinline__ bool ph_restrict3d(const Hier<T>& Hc, int l, const Ctx& c, unsigned char* dyn) {
  using L = SwSlot<T>;
  const Hier<T>& H = Hc;
  const Op<T>& o = H.op[l];
  const Op<T>& co = H.op[l + 1];
  const SweepLev<T>& sw = H.sw[l];
  const int nw = c.gsize - 1, w = c.gcta - 1;
  const int n2 = o.n[2];
  const int ntot = sw.nitems + sw.n1items;
  const int K = (w >= 0 && ntot > w) ? (ntot - 1 - w) / nw + 1 : 0;
  unsigned long long* bars = (unsigned long long*)dyn;
  volatile int* sfail = (volatile int*)(dyn + 8 * SW_NS);
  unsigned char* ring = sw_ring(dyn);
  const unsigned bar0 = smem_u32(bars);
  bool ok = true;
  if (K > 0) {
    if (threadIdx.x == 0) {
      for (int s = 0; s < SW_NS; ++s) mbar_init(bar0 + 8 * s, 1);
      fence_mbar_init();
      *sfail = 0;
    }
    __syncthreads();
    const unsigned char* maps = (const unsigned char*)sw.maps;
    SwIssue<T> iss;
    if (threadIdx.x == 0) {
      iss.start(sw, n2, w, nw, K, maps, 2);
      fence_async_global();
      iss.run(sw, n2, w, nw, maps, ring, bar0, SW_NS, 2);
    }
    // thread t: fine cells (2 cx + h, 2 cy + v), v = 0, 1, of coarse cell
    // (cx, cy) = ((t >> 1) & 15, t >> 5) in both planes of a step
    const int t = threadIdx.x;
    const int hx = t & 1, ccx = (t >> 1) & 15, ccy = t >> 5;
    const bool tin = ccy < (SW_TY >> 1);
    const T scale = T(1) / T(8);
    const int cn0 = co.n[0], cn1 = co.n[1];
    int qb = 0, waited = 0;
    for (int k = 0; k < K && ok; ++k) {
      SwItem<T> it;
      it.at(sw, n2, w + k * nw);
      const SwGrid<T> g(o, it.p);
      const int p = it.p;
      const unsigned pbit = 1u << p;
      const int x0 = it.x0, y0 = it.y0, z0 = it.z0, z1 = it.z1;
      const int G = (z1 - z0 + 4) >> 1, S = (z1 - z0) >> 1;
      T* const cb = co.b[p];
      T* const cx = co.x[p];
      // copies s, s + 1, s + 2 hold planes z0 + 2s - 2 .. z0 + 2s + 3
      int sl0 = qb % SW_NS, sl1 = (qb + 1) % SW_NS, sl2 = (qb + 2) % SW_NS;
      for (int s = 0; s < S; ++s) {
        if (!sw_wait_upto(bar0, waited, qb + min(s + 2, G - 1))) *sfail = 1;
        const unsigned char* const C0 = ring + sl0 * L::BYTES;
        const unsigned char* const C1 = ring + sl1 * L::BYTES;
        const unsigned char* const C2 = ring + sl2 * L::BYTES;
        T acc = T(0);
        if (tin) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            // plane z0 + 2s (copy s + 1, first) then z0 + 2s + 1 (copy s + 1, second)
            const int z = z0 + 2 * s + h;
            const unsigned char* const Pc = C1 + h * L::XB;
            const unsigned char* const Pm = h == 0 ? C0 + L::XB : C1;
            const unsigned char* const Pp = h == 0 ? C1 + L::XB : C2;
            const T* Xc = (const T*)Pc;
            const T* Xm = (const T*)Pm;
            const T* Xp = (const T*)Pp;
            const T* B = (const T*)(Pc + 2 * L::XB);
            const unsigned char* F = C1 + 4 * L::XB + h * L::FB;
            const bool kin = z > 0 && z < n2 - 1;
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              const int rx = 2 * ccx + hx, ry = 2 * ccy + v;
              const int i = x0 + rx, j = y0 + ry;
              if (i >= g.n0 || j >= g.n1) continue;
              const int ly = SW_HY + ry, lx = SW_HX + rx;
              const unsigned f = F[ly * SW_FBX + lx + (SW_FHX - SW_HX)];
              if (!(f & pbit)) continue;
              if (f & F_IRR) {
                const long long cc = ((long long)z * g.n1 + j) * g.n0 + i;
                acc += o.tmp[2 * (long long)o.irr_of_cell[cc] + p];
                continue;
              }
              acc += sw_resid(g, Xc, Xm, Xp, B, i, j, z, kin, lx, ly);
            }
          }
        }
        // the pair of x neighbours of one coarse cell sits in lanes t, t ^ 1
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (tin && hx == 0) {
          const int ci = (x0 >> 1) + ccx, cj = (y0 >> 1) + ccy, ck = (z0 >> 1) + s;
          if (ci < cn0 && cj < cn1 && cb) {
            const long long C = ((long long)ck * cn1 + cj) * cn0 + ci;
            cb[C] = ((co.flags[C] >> p) & 1u) ? acc * scale : T(0);
            cx[C] = T(0);
          }
        }
        __syncthreads();
        if (*sfail) {
          ok = false;
          break;
        }
        // copies below s + 1 (all of the item's after its last step) are read
        // by no later step: refill their slots
        if (t == 0) iss.run(sw, n2, w, nw, maps, ring, bar0, qb + (s == S - 1 ? G : s + 1) + SW_NS, 2);
        sl0 = sl1;
        sl1 = sl2;
        sl2 = sl2 + 1 == SW_NS ? 0 : sl2 + 1;
      }
      qb += G;
    }
    if (!ok) sw_drain(c, bar0, waited, t == 0 ? iss.iq : 0);
    __syncthreads();
    if (t == 0)
      for (int s = 0; s < SW_NS; ++s) mbar_inval(bar0 + 8 * s);
  }
  __syncthreads();
  return ok;
}

}  // namespace ebp
