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

// Relaxes one cell (i, j, k) at box position (lx, ly) of the ring slots sm
// (plane k - 1), s0 (plane k), sp (plane k + 1) when it is a regular cell of
// the level: the implicit stencil of reg_stencil, with the same terms in the
// same order.  Cells off the grid, cut cells and cells without an unknown
// are left alone.
template <class T>
__device__ __forceinline__ void sw_relax(const Op<T>& o, unsigned char* ring, const SweepSlot<T>& L, int two, int i,
                                         int j, int k, int lx, int ly, int sm, int s0, int sp) {
  if ((unsigned)i >= (unsigned)o.n[0] || (unsigned)j >= (unsigned)o.n[1]) return;
  const unsigned char* F = ring + s0 * L.bytes + (two ? 4 : 2) * L.xb;
  const unsigned f = F[ly * SW_FBX + lx + (SW_FHX - SW_HX)] & 7u;
  if (f != 1u && f != 2u) return;  // regular: exactly one phase, no sparse row
  const int p = (int)f - 1;
  const int xo = p * L.xb, bo = (two ? 2 : 1) * L.xb + p * L.xb;
  T* Xc = (T*)(ring + s0 * L.bytes + xo);
  const T* Xm = (const T*)(ring + sm * L.bytes + xo);
  const T* Xp = (const T*)(ring + sp * L.bytes + xo);
  const T bc = ((const T*)(ring + s0 * L.bytes + bo))[ly * SW_BX + lx];
  const int e = ly * SW_BX + lx;
  if (i > 0 && i < o.n[0] - 1 && j > 0 && j < o.n[1] - 1 && k > 0 && k < o.n[2] - 1) {
    const T sum = ((((Xc[e - 1] + Xc[e + 1]) + Xc[e - SW_BX]) + Xc[e + SW_BX]) + Xm[e]) + Xp[e];
    Xc[e] = (o.h2e[p] * bc + sum) * inv_count(6, T(0));
    return;
  }
  const T third = T(1) / T(3);
  T sum = T(0);
  int dg = 0;
  if (i > 0) {
    sum += Xc[e - 1];
    dg += 1;
  } else if (o.bc[0]) {
    sum += Xc[e + 1] * third;
    dg += 3;
  }
  if (i < o.n[0] - 1) {
    sum += Xc[e + 1];
    dg += 1;
  } else if (o.bc[1]) {
    sum += Xc[e - 1] * third;
    dg += 3;
  }
  if (j > 0) {
    sum += Xc[e - SW_BX];
    dg += 1;
  } else if (o.bc[2]) {
    sum += Xc[e + SW_BX] * third;
    dg += 3;
  }
  if (j < o.n[1] - 1) {
    sum += Xc[e + SW_BX];
    dg += 1;
  } else if (o.bc[3]) {
    sum += Xc[e - SW_BX] * third;
    dg += 3;
  }
  if (k > 0) {
    sum += Xm[e];
    dg += 1;
  } else if (o.bc[4]) {
    sum += Xp[e] * third;
    dg += 3;
  }
  if (k < o.n[2] - 1) {
    sum += Xp[e];
    dg += 1;
  } else if (o.bc[5]) {
    sum += Xm[e] * third;
    dg += 3;
  }
  Xc[e] = (o.h2e[p] * bc + sum) * inv_count(dg, T(0));
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
  const long long sxy = (long long)n0 * n1;
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
    // the ring's red cells (2 rows of 17, one per tile row) by t < ty + 34
    const int t = threadIdx.x;
    const int tr = t >> 4, tm = t & 15;
    const bool tin = t < 16 * ty;
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
        const int sm2 = (q0 - 2) & (SW_NS - 1), sm = (q0 - 1) & (SW_NS - 1), s0 = q0 & (SW_NS - 1),
                  sp = (q0 + 1) & (SW_NS - 1);
        // red cells of plane zs on the tile and its one-cell ring
        if (zs <= z1 && zs >= 0 && zs < n2) {
          if (tin) {
            const int j = y0 + tr;
            const int lx = SW_HX + ((j + zs) & 1) + 2 * tm;
            sw_relax(o, ring, L, two, x0 - SW_HX + lx, j, zs, lx, SW_HY + tr, sm, s0, sp);
          }
          if (t < ty + 34) {
            int j, lx, ly;
            if (t < 34) {  // ring rows above and below the tile
              ly = t < 17 ? SW_HY - 1 : SW_HY + ty;
              j = y0 - SW_HY + ly;
              lx = SW_HX - 1 + ((j + zs + 1) & 1) + 2 * (t < 17 ? t : t - 17);
            } else {  // the ring cell at the left or right end of a tile row
              ly = SW_HY + t - 34;
              j = y0 - SW_HY + ly;
              lx = ((j + zs) & 1) ? SW_HX - 1 : SW_HX + SW_TX;
            }
            sw_relax(o, ring, L, two, x0 - SW_HX + lx, j, zs, lx, ly, sm, s0, sp);
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
          sw_relax(o, ring, L, two, x0 - SW_HX + lx, j, zw, lx, SW_HY + tr, sm2, sm, s0);
        }
        // store plane zs - 2: the tile's unknowns, both colours, cut cells as given
        const int zo = zs - 2;
        if (zo >= z0 && zo < z1) {
          const int so = (q0 - 2 - 0) & (SW_NS - 1);
          const unsigned char* F = ring + ((q0 - 2) & (SW_NS - 1)) * L.bytes + (two ? 4 : 2) * L.xb;
          (void)so;
          const int h1w = slot1[(q0 - 2) & (SW_NS - 1)];
          const T* X0 = (const T*)(ring + ((q0 - 2) & (SW_NS - 1)) * L.bytes);
          for (int idx = t; idx < SW_TX * ty; idx += blockDim.x) {
            const int ry = idx >> 5, rx = idx & 31;
            const int i = x0 + rx, j = y0 + ry;
            if (i >= n0 || j >= n1) continue;
            const int ly = SW_HY + ry, lx = SW_HX + rx;
            const unsigned f = F[ly * SW_FBX + lx + (SW_FHX - SW_HX)];
            const long long cc = (long long)zo * sxy + (long long)j * n0 + i;
            const int e = ly * SW_BX + lx;
            if (f & 1u) sw.alt[0][cc] = X0[e];
            if ((f & 2u) && h1w) sw.alt[1][cc] = ((const T*)((const unsigned char*)X0 + L.xb))[e];
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

}  // namespace ebp
