// sweep3d.cuh -- one red-black Gauss-Seidel sweep of a large 3D level in a
// single pass over memory (arXiv:1809.03745, Sec. 3.3.2 smooths by
// multi-colour Gauss-Seidel; the order of the colours within a sweep is a
// free choice of the multigrid, not of the discretisation).
//
// A classic colour pass reads the whole level and writes half of it, so a
// sweep moves about twice the bytes the method needs.  Here a CTA owns an
// x-y tile of 32 x TY cells and streams it along z through shared memory:
// TMA (cp.async.bulk.tensor) brings in, per plane, the tile with a halo of
// x, b and the cell flags, several planes ahead of use, each plane completing
// an mbarrier.  At step zs the CTA relaxes the red regular cells of plane zs
// on the tile plus a one-cell ring (reading black values of planes zs-1..zs+1,
// not yet updated), then the black regular cells of plane zs-1 on the tile
// (reading the new red values of planes zs-2..zs), then stores plane zs-1.
// The ring's red values equal those the neighbouring tile computes, because
// every read comes from the previous iterate: the sweep is out of place,
// x -> alt, and the two buffers swap roles afterwards.  Cut cells (sparse
// rows) are not touched here: their new values were written into x before
// the sweep, so the regular cells already see them.
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

// byte offsets of one ring slot's buffers (x[0], x[1], b[0], b[1], flags),
// each a multiple of 128 bytes
template <class T>
struct SweepSlot {
  int xb, fb, bytes;  // bytes of one x or b box, of the flags box, of the slot
  __device__ __host__ SweepSlot(int ty, int two) {
    const int by = ty + 2 * SW_HY;
    xb = SW_BX * by * (int)sizeof(T);
    fb = SW_FBX * by;
    bytes = (two ? 4 : 2) * xb + fb;
  }
};

// The level's constants, held in registers for the streamed passes (the
// hierarchy itself sits in shared memory, where every field read is a load).
template <class T>
struct SwGrid {
  int n0, n1, n2;
  unsigned bcm;          // bit s set: Dirichlet wall on side s (xlo, xhi, ylo, yhi, zlo, zhi)
  T h2e0, h2e1, ceps0, ceps1;
  int xb, fo, bo;        // bytes of an x/b box, offset of the flags box, of phase 0's b box
  int slot;              // bytes of a ring slot
  __device__ SwGrid(const Op<T>& o, const SweepSlot<T>& L, int two) {
    n0 = o.n[0];
    n1 = o.n[1];
    n2 = o.n[2];
    bcm = 0u;
    for (int q = 0; q < 6; ++q) bcm |= (o.bc[q] ? 1u : 0u) << q;
    h2e0 = o.h2e[0];
    h2e1 = o.h2e[1];
    ceps0 = o.ceps[0];
    ceps1 = o.ceps[1];
    xb = L.xb;
    fo = (two ? 4 : 2) * L.xb;
    bo = (two ? 2 : 1) * L.xb;
    slot = L.bytes;
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

// Relaxes cell (i, j, k) at box position (lx, ly) of the planes P0 (k), Pm
// (k - 1), Pp (k + 1) when it is a regular cell of the level; kin: k is not
// on a wall plane.  Cells off the grid, cut cells and cells without an
// unknown are left alone.
template <class T>
__device__ __forceinline__ void sw_relax(const SwGrid<T>& g, unsigned char* P0, const unsigned char* Pm,
                                         const unsigned char* Pp, int i, int j, int k, bool kin, int lx, int ly) {
  if ((unsigned)i >= (unsigned)g.n0 || (unsigned)j >= (unsigned)g.n1) return;
  const unsigned f = P0[g.fo + ly * SW_FBX + lx + (SW_FHX - SW_HX)] & 7u;
  if (f - 1u > 1u) return;  // regular: exactly one phase, no sparse row
  const int po = f == 2u ? g.xb : 0;
  T* Xc = (T*)(P0 + po);
  const T* Xm = (const T*)(Pm + po);
  const T* Xp = (const T*)(Pp + po);
  const int e = ly * SW_BX + lx;
  const T bcell = ((const T*)(P0 + g.bo + po))[e];
  const T h2e = f == 2u ? g.h2e1 : g.h2e0;
  if (kin && (unsigned)(i - 1) < (unsigned)(g.n0 - 2) && (unsigned)(j - 1) < (unsigned)(g.n1 - 2)) {
    const T sum = ((((Xc[e - 1] + Xc[e + 1]) + Xc[e - SW_BX]) + Xc[e + SW_BX]) + Xm[e]) + Xp[e];
    Xc[e] = (h2e * bcell + sum) * inv_count(6, T(0));
    return;
  }
  T sum;
  int dg;
  sw_wall_stencil(g, Xm, Xc, Xp, e, i, j, k, sum, dg);
  Xc[e] = (h2e * bcell + sum) * inv_count(dg, T(0));
}

// One fused pass over the regular cells of grid level l (SweepLev on),
// x -> alt, then x and alt swap in this CTA's copy of the hierarchy.  CTA 0
// of the group keeps the coarse levels in its shared memory and sits the
// pass out; the other CTAs take the tiles round-robin.  `dyn` is the
// dynamic shared memory.
//
// Step zs of an item: wait for plane zs + 1; red cells of plane zs (tile
// and ring); one block barrier; black cells of plane zs - 1 (tile); store
// plane zs - 2, final since the barrier; refill the slot of plane zs - 3,
// which nothing reads any more.  The ring has SW_NS slots: four planes in
// use, four in flight.
template <class T>
__device__ bool ph_sweep3d(const Hier<T>& Hc, int l, const Ctx& c, unsigned char* dyn) {
  Hier<T>& H = const_cast<Hier<T>&>(Hc);
  Op<T>& o = H.op[l];
  SweepLev<T>& sw = H.sw[l];
  const int two = o.x[1] != nullptr;
  const int ty = sw.ty;
  const SweepSlot<T> L(ty, two);
  const int nw = c.gsize - 1, w = c.gcta - 1;
  const int n0 = o.n[0], n1 = o.n[1], n2 = o.n[2];
  const int K = (w >= 0 && sw.nitems > w) ? (sw.nitems - 1 - w) / nw + 1 : 0;
  // layout: SW_NS mbarriers, item mask words, SW_NS has1 flags, a fail flag, then the ring
  unsigned long long* bars = (unsigned long long*)dyn;
  unsigned* mask = (unsigned*)(dyn + 8 * SW_NS_MAX);
  int* slot1 = (int*)(dyn + 8 * SW_NS_MAX + 4 * SW_MASK_MAX);
  volatile int* sfail = slot1 + SW_NS_MAX;
  // the ring starts on a 128-byte boundary of the shared window (the host
  // reserves 128 bytes of slack for this)
  unsigned char* ring = dyn + SW_HEAD + ((128u - (smem_u32(dyn + SW_HEAD) & 127u)) & 127u);
  const unsigned bar0 = smem_u32(bars);
  bool ok = true;
  if (K > 0) {
    const int nwords = (sw.nitems + 31) >> 5;
    for (int q = threadIdx.x; q < nwords; q += blockDim.x) mask[q] = two ? sw.has1[q] : 0u;
    if (threadIdx.x == 0) {
      for (int s = 0; s < SW_NS; ++s) mbar_init(bar0 + 8 * s, 1);
      fence_mbar_init();
      *sfail = 0;
    }
    __syncthreads();
    const int ntx = sw.ntx, nty = sw.nty, zc = sw.zc;
    const unsigned char* mp = (const unsigned char*)sw.maps;  // 7 tensor maps of 128 bytes
    const void* mx0 = mp + 128 * (2 * sw.par + 0);
    const void* mx1 = mp + 128 * (2 * sw.par + 1);
    const void* mb0 = mp + 128 * 4;
    const void* mb1 = mp + 128 * 5;
    const void* mf = mp + 128 * 6;
    auto geom = [&](int k, int& x0, int& y0, int& z0, int& z1, int& h1) {
      const int it = w + k * nw;
      const int tx = it % ntx, r = it / ntx;
      x0 = tx * SW_TX;
      y0 = (r % nty) * ty;
      z0 = (r / nty) * zc;
      z1 = min(z0 + zc, n2);
      h1 = (mask[it >> 5] >> (it & 31)) & 1;
    };
    // issue cursor (thread 0): item ik and its geometry, plane index itp, load index iq
    int ik = 0, itp = 0, iq = 0;
    int gx0 = 0, gy0 = 0, gz0 = 0, gz1 = 0, gh1 = 0;
    if (threadIdx.x == 0) geom(0, gx0, gy0, gz0, gz1, gh1);
    auto issue = [&](int limit) {
      while (iq < limit && ik < K) {
        const int s = iq & (SW_NS - 1);
        const unsigned bar = bar0 + 8 * s;
        const unsigned base = smem_u32(ring + s * L.bytes);
        const int z = gz0 - 2 + itp;
        slot1[s] = gh1;
        mbar_expect_tx(bar, (unsigned)((gh1 ? 4 : 2) * L.xb + L.fb));
        tma_load3(base, mx0, gx0 - SW_HX, gy0 - SW_HY, z, bar);
        tma_load3(base + (two ? 2 : 1) * L.xb, mb0, gx0 - SW_HX, gy0 - SW_HY, z, bar);
        if (gh1) {
          tma_load3(base + L.xb, mx1, gx0 - SW_HX, gy0 - SW_HY, z, bar);
          tma_load3(base + 3 * L.xb, mb1, gx0 - SW_HX, gy0 - SW_HY, z, bar);
        }
        tma_load3(base + (two ? 4 : 2) * L.xb, mf, gx0 - SW_FHX, gy0 - SW_HY, z, bar);
        ++iq;
        if (++itp == gz1 - gz0 + 4) {
          itp = 0;
          if (++ik < K) geom(ik, gx0, gy0, gz0, gz1, gh1);
        }
      }
    };
    if (threadIdx.x == 0) {
      fence_async_global();  // x was last written by generic stores of other CTAs
      issue(SW_NS);
    }
    // thread mapping: the tile's cells of one colour, 16 per row (t < 16 ty);
    // the ring's red cells (2 rows of 17, one per tile row) by the last
    // ty + 34 threads, away from warp 0, which issues the loads
    const int t = threadIdx.x;
    const int tr = t >> 4, tm = t & 15;
    const bool tin = t < 16 * ty;
    const int tring = (int)blockDim.x - 1 - t;
    const SwGrid<T> g(o, L, two);
    T* const alt0 = sw.alt[0];
    T* const alt1 = sw.alt[1];
    int qb = 0, waited = 0;
    for (int k = 0; k < K && ok; ++k) {
      int x0, y0, z0, z1, h1;
      geom(k, x0, y0, z0, z1, h1);
      for (int zs = z0 - 1; zs <= z1 + 1; ++zs) {
        // planes up to zs + 1 (the item's last is z1 + 1) have landed
        const int need = qb + min(zs + 1, z1 + 1) - (z0 - 2);
        for (; waited <= need; ++waited)
          if (!mbar_wait(bar0 + 8 * (waited & (SW_NS - 1)), (unsigned)((waited / SW_NS) & 1))) {
            *sfail = 1;
            break;
          }
        const int q0 = qb + zs - z0 + 2;  // load index of plane zs
        unsigned char* const Pm2 = ring + ((q0 - 2) & (SW_NS - 1)) * g.slot;
        unsigned char* const Pm = ring + ((q0 - 1) & (SW_NS - 1)) * g.slot;
        unsigned char* const P0 = ring + (q0 & (SW_NS - 1)) * g.slot;
        unsigned char* const Pp = ring + ((q0 + 1) & (SW_NS - 1)) * g.slot;
        // red cells of plane zs on the tile and its one-cell ring
        if (zs <= z1 && zs >= 0 && zs < n2) {
          const bool kin = zs > 0 && zs < n2 - 1;
          if (tin) {
            const int j = y0 + tr;
            const int lx = SW_HX + ((j + zs) & 1) + 2 * tm;
            sw_relax(g, P0, Pm, Pp, x0 - SW_HX + lx, j, zs, kin, lx, SW_HY + tr);
          }
          if (tring < ty + 34) {
            int j, lx, ly;
            if (tring < 34) {  // ring rows above and below the tile
              ly = tring < 17 ? SW_HY - 1 : SW_HY + ty;
              j = y0 - SW_HY + ly;
              lx = SW_HX - 1 + ((j + zs + 1) & 1) + 2 * (tring < 17 ? tring : tring - 17);
            } else {  // the ring cell at the left or right end of a tile row
              ly = SW_HY + tring - 34;
              j = y0 - SW_HY + ly;
              lx = ((j + zs) & 1) ? SW_HX - 1 : SW_HX + SW_TX;
            }
            sw_relax(g, P0, Pm, Pp, x0 - SW_HX + lx, j, zs, kin, lx, ly);
          }
        }
        fence_async_smem();
        __syncthreads();
        if (*sfail) {
          ok = false;
          break;
        }
        // black cells of plane zs - 1 on the tile
        const int zw = zs - 1;
        if (zw >= z0 && zw < z1 && tin) {
          const int j = y0 + tr;
          const int lx = SW_HX + ((j + zw + 1) & 1) + 2 * tm;
          sw_relax(g, Pm, Pm2, P0, x0 - SW_HX + lx, j, zw, zw > 0 && zw < n2 - 1, lx, SW_HY + tr);
        }
        // store plane zs - 2: the tile's unknowns, both colours, cut cells as given
        const int zo = zs - 2;
        if (zo >= z0 && zo < z1) {
          const unsigned char* F = Pm2 + g.fo;
          const int h1w = slot1[(q0 - 2) & (SW_NS - 1)];
          const T* X0 = (const T*)Pm2;
          const T* X1 = (const T*)(Pm2 + g.xb);
          const int rx = t & 31, i = x0 + rx;
          if (i < n0)
            for (int ry = t >> 5; ry < ty; ry += (int)(blockDim.x >> 5)) {
              const int j = y0 + ry;
              if (j >= n1) break;
              const int ly = SW_HY + ry, lx = SW_HX + rx;
              const unsigned f = F[ly * SW_FBX + lx + (SW_FHX - SW_HX)];
              const long long cc = ((long long)zo * n1 + j) * n0 + i;
              const int e = ly * SW_BX + lx;
              if (f & 1u) alt0[cc] = X0[e];
              if ((f & 2u) && h1w) alt1[cc] = X1[e];
            }
        }
        // the slots of planes up to zs - 3 are free (their last readers ran
        // before the barrier): refill them
        if (t == 0) issue(qb + max(0, zs - z0) + SW_NS);
      }
      qb += z1 - z0 + 4;
    }
    if (!ok) {
      // give up: raise the error word, then let this CTA's copies in flight land
      if (t == 0) {
        atomicOr(c.B.err, 1);
        for (; waited < iq; ++waited)
          if (!mbar_wait(bar0 + 8 * (waited & (SW_NS - 1)), (unsigned)((waited / SW_NS) & 1))) break;
      }
    }
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

// Residual b - A x of the regular cell (i, j, k) at box position (lx, ly) of
// the planes P0 (k), Pm, Pp in phase p (po: its byte offset), with the terms
// and order of cell_residual.
template <class T>
__device__ __forceinline__ T sw_resid(const SwGrid<T>& g, const unsigned char* P0, const unsigned char* Pm,
                                      const unsigned char* Pp, int po, T ceps, int i, int j, int k, bool kin, int lx,
                                      int ly) {
  const T* Xc = (const T*)(P0 + po);
  const T* Xm = (const T*)(Pm + po);
  const T* Xp = (const T*)(Pp + po);
  const int e = ly * SW_BX + lx;
  const T bcell = ((const T*)(P0 + g.bo + po))[e];
  if (kin && (unsigned)(i - 1) < (unsigned)(g.n0 - 2) && (unsigned)(j - 1) < (unsigned)(g.n1 - 2)) {
    const T sum = ((((Xc[e - 1] + Xc[e + 1]) + Xc[e - SW_BX]) + Xc[e + SW_BX]) + Xm[e]) + Xp[e];
    return bcell - ceps * ((T)6 * Xc[e] - sum);
  }
  T sum;
  int dg;
  sw_wall_stencil(g, Xm, Xc, Xp, e, i, j, k, sum, dg);
  return bcell - ceps * ((T)dg * Xc[e] - sum);
}

// Residual + restriction of grid level l (SweepLev on) onto level l + 1
// (half the cells per axis): coarse b = mean of the children's residuals
// (cut children from the sparse residual rows in tmp), coarse x = 0.  The
// level streams through the same ring as the sweep; a step computes the
// residuals of one plane, pairs of x neighbours combine by a shuffle and
// pairs of planes in registers, and the coarse plane is stored after the
// odd one.  One block barrier per step.
template <class T>
__device__ bool ph_restrict3d(const Hier<T>& Hc, int l, const Ctx& c, unsigned char* dyn) {
  const Hier<T>& H = Hc;
  const Op<T>& o = H.op[l];
  const Op<T>& co = H.op[l + 1];
  const SweepLev<T>& sw = H.sw[l];
  const int two = o.x[1] != nullptr;
  const int ty = sw.ty;
  const SweepSlot<T> L(ty, two);
  const int nw = c.gsize - 1, w = c.gcta - 1;
  const int n0 = o.n[0], n1 = o.n[1], n2 = o.n[2];
  const int K = (w >= 0 && sw.nitems > w) ? (sw.nitems - 1 - w) / nw + 1 : 0;
  unsigned long long* bars = (unsigned long long*)dyn;
  unsigned* mask = (unsigned*)(dyn + 8 * SW_NS_MAX);
  int* slot1 = (int*)(dyn + 8 * SW_NS_MAX + 4 * SW_MASK_MAX);
  volatile int* sfail = slot1 + SW_NS_MAX;
  unsigned char* ring = dyn + SW_HEAD + ((128u - (smem_u32(dyn + SW_HEAD) & 127u)) & 127u);
  const unsigned bar0 = smem_u32(bars);
  bool ok = true;
  if (K > 0) {
    const int nwords = (sw.nitems + 31) >> 5;
    for (int q = threadIdx.x; q < nwords; q += blockDim.x) mask[q] = two ? sw.has1[q] : 0u;
    if (threadIdx.x == 0) {
      for (int s = 0; s < SW_NS; ++s) mbar_init(bar0 + 8 * s, 1);
      fence_mbar_init();
      *sfail = 0;
    }
    __syncthreads();
    const int ntx = sw.ntx, nty = sw.nty, zc = sw.zc;
    const unsigned char* mp = (const unsigned char*)sw.maps;
    const void* mx0 = mp + 128 * (2 * sw.par + 0);
    const void* mx1 = mp + 128 * (2 * sw.par + 1);
    const void* mb0 = mp + 128 * 4;
    const void* mb1 = mp + 128 * 5;
    const void* mf = mp + 128 * 6;
    auto geom = [&](int k, int& x0, int& y0, int& z0, int& z1, int& h1) {
      const int it = w + k * nw;
      const int tx = it % ntx, r = it / ntx;
      x0 = tx * SW_TX;
      y0 = (r % nty) * ty;
      z0 = (r / nty) * zc;
      z1 = min(z0 + zc, n2);
      h1 = (mask[it >> 5] >> (it & 31)) & 1;
    };
    // loads: planes z0 - 1 .. z1 of each item
    int ik = 0, itp = 0, iq = 0;
    int gx0 = 0, gy0 = 0, gz0 = 0, gz1 = 0, gh1 = 0;
    if (threadIdx.x == 0) geom(0, gx0, gy0, gz0, gz1, gh1);
    auto issue = [&](int limit) {
      while (iq < limit && ik < K) {
        const int s = iq & (SW_NS - 1);
        const unsigned bar = bar0 + 8 * s;
        const unsigned base = smem_u32(ring + s * L.bytes);
        const int z = gz0 - 1 + itp;
        slot1[s] = gh1;
        mbar_expect_tx(bar, (unsigned)((gh1 ? 4 : 2) * L.xb + L.fb));
        tma_load3(base, mx0, gx0 - SW_HX, gy0 - SW_HY, z, bar);
        tma_load3(base + (two ? 2 : 1) * L.xb, mb0, gx0 - SW_HX, gy0 - SW_HY, z, bar);
        if (gh1) {
          tma_load3(base + L.xb, mx1, gx0 - SW_HX, gy0 - SW_HY, z, bar);
          tma_load3(base + 3 * L.xb, mb1, gx0 - SW_HX, gy0 - SW_HY, z, bar);
        }
        tma_load3(base + (two ? 4 : 2) * L.xb, mf, gx0 - SW_FHX, gy0 - SW_HY, z, bar);
        ++iq;
        if (++itp == gz1 - gz0 + 2) {
          itp = 0;
          if (++ik < K) geom(ik, gx0, gy0, gz0, gz1, gh1);
        }
      }
    };
    if (threadIdx.x == 0) {
      fence_async_global();  // x was last written by generic stores of other CTAs
      issue(SW_NS);
    }
    // thread t: fine cells (2 cx + h, 2 cy + v) of coarse cell (cx, cy), h = t & 1,
    // for the plane's two child rows v = 0, 1; coarse cells 16 per row
    const int t = threadIdx.x;
    const int hx = t & 1, ccx = (t >> 1) & 15, ccy = t >> 5;
    const bool tin = ccy < (ty >> 1);
    const SwGrid<T> g(o, L, two);
    const T scale = T(1) / T(8);
    const int cn0 = co.n[0], cn1 = co.n[1];
    const long long csxy = (long long)cn0 * cn1;
    int qb = 0, waited = 0;
    T acc[2] = {T(0), T(0)};
    for (int k = 0; k < K && ok; ++k) {
      int x0, y0, z0, z1, h1;
      geom(k, x0, y0, z0, z1, h1);
      for (int zs = z0; zs < z1; ++zs) {
        const int need = qb + zs + 1 - (z0 - 1);
        for (; waited <= need; ++waited)
          if (!mbar_wait(bar0 + 8 * (waited & (SW_NS - 1)), (unsigned)((waited / SW_NS) & 1))) {
            *sfail = 1;
            break;
          }
        const int q0 = qb + zs - (z0 - 1);
        const unsigned char* const Pm = ring + ((q0 - 1) & (SW_NS - 1)) * g.slot;
        const unsigned char* const P0 = ring + (q0 & (SW_NS - 1)) * g.slot;
        const unsigned char* const Pp = ring + ((q0 + 1) & (SW_NS - 1)) * g.slot;
        const unsigned char* F = P0 + g.fo;
        const int h1s = slot1[q0 & (SW_NS - 1)];
        const bool kin = zs > 0 && zs < n2 - 1;
        if (tin) {
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int rx = 2 * ccx + hx, ry = 2 * ccy + v;
            const int i = x0 + rx, j = y0 + ry;
            if (i >= n0 || j >= n1) continue;
            const int ly = SW_HY + ry, lx = SW_HX + rx;
            const unsigned f = F[ly * SW_FBX + lx + (SW_FHX - SW_HX)];
            if (!(f & 3u)) continue;
            if (f & F_IRR) {
              const long long cc = ((long long)zs * n1 + j) * n0 + i;
              const long long r2 = 2 * (long long)o.irr_of_cell[cc];
              if (f & 1u) acc[0] += o.tmp[r2];
              if (f & 2u) acc[1] += o.tmp[r2 + 1];
              continue;
            }
            if (f & 1u) {
              acc[0] += sw_resid(g, P0, Pm, Pp, 0, g.ceps0, i, j, zs, kin, lx, ly);
            } else if (h1s) {  // (a box without dielectric unknowns has no phase-1 cell)
              acc[1] += sw_resid(g, P0, Pm, Pp, g.xb, g.ceps1, i, j, zs, kin, lx, ly);
            }
          }
        }
        // after the odd plane: the pair of x neighbours of one coarse cell sits
        // in lanes t, t ^ 1 (each lane holds its column of both planes)
        if ((zs & 1) == 1) {
          acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
          acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], 1);
        }
        if ((zs & 1) == 1 && tin && hx == 0) {
          const int ci = (x0 >> 1) + ccx, cj = (y0 >> 1) + ccy, ck = zs >> 1;
          if (ci < cn0 && cj < cn1) {
            const long long C = (long long)ck * csxy + (long long)cj * cn0 + ci;
            const unsigned cfl = co.flags[C];
            for (int p = 0; p < 2; ++p) {
              if (co.b[p] == nullptr) continue;
              co.b[p][C] = ((cfl >> p) & 1u) ? acc[p] * scale : T(0);
              co.x[p][C] = T(0);
            }
          }
        }
        if ((zs & 1) == 1) acc[0] = acc[1] = T(0);
        __syncthreads();
        if (*sfail) {
          ok = false;
          break;
        }
        // plane zs - 1 is read by no later step: its slot takes the next load
        if (t == 0) issue(q0 - 1 + 1 + SW_NS);
      }
      qb += z1 - z0 + 2;
    }
    if (!ok) {
      if (t == 0) {
        atomicOr(c.B.err, 1);
        for (; waited < iq; ++waited)
          if (!mbar_wait(bar0 + 8 * (waited & (SW_NS - 1)), (unsigned)((waited / SW_NS) & 1))) break;
      }
    }
    __syncthreads();
    if (t == 0)
      for (int s = 0; s < SW_NS; ++s) mbar_inval(bar0 + 8 * s);
  }
  __syncthreads();
  return ok;
}

}  // namespace ebp
