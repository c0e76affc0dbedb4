// tagging.cu -- refinement tags of Sec. 6 and the box a regrid step takes
// from them.
//
// The tracer is T = |E| / max |E|; a cell is tagged for refinement when
// |grad T| dx / T > eps1 or T > eps2 and for coarsening when
// |grad T| dx / T < eps3 and T < eps4.  Three passes over the grid: the first
// writes |E| per cell into a scratch array and takes its maximum (order-free
// atomicMax on the bit pattern of a non-negative double), the second divides
// by the maximum in place, the third reads T at the cell and its axis
// neighbours, forms the gradient by centred or one-sided differences in
// index units (dx cancels), the tag byte, and the bounding box and count of
// the marked cells (warp reductions, then one atomic per warp).  FP64 is slow
// on this part, so every square root and division is taken once per cell
// (reading the neighbours' T instead of recomputing them costs 8 bytes each,
// mostly from L1).  Every product and sum is written with round-to-nearest
// intrinsics (this unit is also compiled without FMA contraction) and sqrt
// and division are correctly rounded, so the tags are a function of E alone
// and match a plain FP64 evaluation in the same order.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstring>
#include <string>

#include "eb_internal.h"

using namespace ebp;

namespace {

constexpr int TBT = 256;
int nbt(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + TBT - 1) / TBT, 152LL * 16)); }

struct TagOut {
  unsigned long long emax;  // bit pattern of max |E|
  unsigned long long count;
  int lo[3], hi[3];  // hi inclusive while reducing
};

struct TagView {
  int D;
  int n[3];
  long long ncell;
  const uint8_t* flags;
  const double* E;  // [D][2][ncell]
};

// largest field magnitude over the phases with an unknown (0 where covered)
__device__ __forceinline__ double cell_mag(const TagView& v, long long c) {
  const unsigned f = v.flags[c];
  double mag = 0.0;
  for (int p = 0; p < 2; ++p) {
    if (!((f >> p) & 1u)) continue;  // a phase without an unknown is never selected: skip its reads
    const double e0 = v.E[(long long)p * v.ncell + c];
    double m2 = __dmul_rn(e0, e0);
    for (int a = 1; a < v.D; ++a) {
      const double e = v.E[((long long)a * 2 + p) * v.ncell + c];
      m2 = __dadd_rn(m2, __dmul_rn(e, e));
    }
    const double m = sqrt(m2);
    if (m > mag) mag = m;
  }
  return mag;
}

__global__ void k_emag(TagView v, double* T, TagOut* out) {
  double m = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < v.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const double mc = cell_mag(v, c);
    T[c] = mc;
    m = fmax(m, mc);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(&out->emax, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_tnorm(long long n, double* T, const TagOut* out) {
  const double emax = __longlong_as_double((long long)out->emax);
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    T[c] = emax > 0.0 ? T[c] / emax : 0.0;
}

template <int D>
__global__ void k_tag(TagView v, const double* __restrict__ Tt, double eps1, double eps2, double eps3, double eps4,
                      int keep, int klo0, int klo1, int klo2, int khi0, int khi1, int khi2, uint8_t* tags,
                      TagOut* out) {
  const int klo[3] = {klo0, klo1, klo2}, khi[3] = {khi0, khi1, khi2};
  int mlo[3] = {INT_MAX, INT_MAX, INT_MAX}, mhi[3] = {-1, -1, -1};
  unsigned cnt = 0;
  const long long stride[3] = {1, v.n[0], (long long)v.n[0] * v.n[1]};
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < v.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const unsigned r = (unsigned)(c / v.n[0]);
    const int I[3] = {(int)(c - (long long)r * v.n[0]), (int)(r % (unsigned)v.n[1]), (int)(r / (unsigned)v.n[1])};
    uint8_t t = 0;
    if (v.flags[c] & 3u) {
      const double T = Tt[c];
      double s2 = 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const bool hp = I[a] + 1 < v.n[a] && (v.flags[c + stride[a]] & 3u);
        const bool hm = I[a] > 0 && (v.flags[c - stride[a]] & 3u);
        const double Tp = hp ? Tt[c + stride[a]] : 0.0;
        const double Tm = hm ? Tt[c - stride[a]] : 0.0;
        const double d = hp && hm ? __dmul_rn(__dsub_rn(Tp, Tm), 0.5) : hp ? __dsub_rn(Tp, T)
                                                                      : hm ? __dsub_rn(T, Tm) : 0.0;
        s2 = __dadd_rn(s2, __dmul_rn(d, d));
      }
      const double g = sqrt(s2);
      const double ratio = T > 0.0 ? g / T : (g > 0.0 ? INFINITY : 0.0);
      const bool refine = ratio > eps1 || T > eps2;
      const bool coarsen = ratio < eps3 && T < eps4;
      t = (refine ? 1 : 0) | (coarsen ? 2 : 0);
      bool marked = refine;
      if (!marked && keep && !coarsen) {
        marked = true;
#pragma unroll
        for (int a = 0; a < D; ++a) marked = marked && I[a] >= klo[a] && I[a] < khi[a];
      }
      if (marked) {
        ++cnt;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          mlo[a] = min(mlo[a], I[a]);
          mhi[a] = max(mhi[a], I[a]);
        }
      }
    }
    if (tags) tags[c] = t;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mlo[a] = __reduce_min_sync(0xffffffffu, mlo[a]);
    mhi[a] = __reduce_max_sync(0xffffffffu, mhi[a]);
  }
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) {
    atomicAdd(&out->count, (unsigned long long)cnt);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(&out->lo[a], mlo[a]);
      atomicMax(&out->hi[a], mhi[a]);
    }
  }
}

}  // namespace

extern "C" eb_status eb_tag_cells(const eb_geom* G, const double* d_E, const double eps[4], const int* keep_lo,
                                  const int* keep_hi, unsigned char* d_tags, int bbox_lo[3], int bbox_hi[3],
                                  long long* n_marked, double* e_max, void* stream) {
  if (!G || !d_E || !eps || !bbox_lo || !bbox_hi || !n_marked || (!keep_lo) != (!keep_hi)) {
    set_error("null argument (keep_lo and keep_hi go together)");
    return EB_ERR_INVALID;
  }
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(eps[k])) {
      set_error("tagging thresholds must be finite");
      return EB_ERR_INVALID;
    }
  // the geometry's arrays live on the device it was built on: the kernels
  // must run there
  int dev = -1;
  cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess) return cuda_fail(ed, "device query");
  if (dev != G->device) {
    set_error("the current device (" + std::to_string(dev) + ") is not the geometry's device (" +
              std::to_string(G->device) + ")");
    return EB_ERR_INVALID;
  }
  const DevLevel& F = G->L[0];
  TagView v;
  v.D = F.g.D;
  for (int k = 0; k < 3; ++k) v.n[k] = k < v.D ? F.g.n[k] : 1;
  v.ncell = F.g.ncell;
  v.flags = F.flags;
  v.E = d_E;
  cudaStream_t s = (cudaStream_t)stream;
  TagOut init;
  std::memset(&init, 0, sizeof(init));
  for (int a = 0; a < 3; ++a) {
    init.lo[a] = INT_MAX;
    init.hi[a] = -1;
  }
  // one allocation: the result words, then T [ncell] (16-byte aligned)
  const size_t head = (sizeof(TagOut) + 255) / 256 * 256;
  char* d_buf = nullptr;
  cudaError_t e = cudaMalloc(&d_buf, head + sizeof(double) * (size_t)v.ncell);
  if (e != cudaSuccess) return cuda_fail(e, "tag scratch");
  TagOut* d_out = (TagOut*)d_buf;
  double* d_T = (double*)(d_buf + head);
  e = cudaMemcpyAsync(d_out, &init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_emag<<<nbt(v.ncell), TBT, 0, s>>>(v, d_T, d_out);
    k_tnorm<<<nbt(v.ncell), TBT, 0, s>>>(v.ncell, d_T, d_out);
    note_launch(2);
    const int keep = keep_lo ? 1 : 0;
    int klo[3] = {0, 0, 0}, khi[3] = {0, 0, 0};
    if (keep)
      for (int a = 0; a < 3; ++a) {
        klo[a] = keep_lo[a];
        khi[a] = keep_hi[a];
      }
    if (v.D == 2)
      k_tag<2><<<nbt(v.ncell), TBT, 0, s>>>(v, d_T, eps[0], eps[1], eps[2], eps[3], keep, klo[0], klo[1], klo[2],
                                            khi[0], khi[1], khi[2], d_tags, d_out);
    else
      k_tag<3><<<nbt(v.ncell), TBT, 0, s>>>(v, d_T, eps[0], eps[1], eps[2], eps[3], keep, klo[0], klo[1], klo[2],
                                            khi[0], khi[1], khi[2], d_tags, d_out);
    note_launch();
    e = cudaGetLastError();
  }
  TagOut res;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&res, d_out, sizeof(res), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_buf);
  if (e != cudaSuccess) return cuda_fail(e, "refinement tags");
  *n_marked = (long long)res.count;
  for (int a = 0; a < 3; ++a) {
    bbox_lo[a] = res.count ? res.lo[a] : 0;
    bbox_hi[a] = res.count ? res.hi[a] + 1 : 0;
  }
  if (e_max) {
    unsigned long long b = res.emax;
    std::memcpy(e_max, &b, sizeof(double));
  }
  return EB_OK;
}

extern "C" eb_status eb_regrid_box(int dim, const int n[3], const int cf_lo[3], const int cf_hi[3],
                                   const int bbox_lo[3], const int bbox_hi[3], long long n_marked, int buf, int block,
                                   int box_lo[3], int box_hi[3], int* has_box) {
  if (!n || !cf_lo || !cf_hi || !bbox_lo || !bbox_hi || !box_lo || !box_hi || !has_box || dim < 2 || dim > 3 ||
      buf < 0 || block < 1) {
    set_error("invalid argument");
    return EB_ERR_INVALID;
  }
  *has_box = 0;
  for (int a = 0; a < 3; ++a) {
    box_lo[a] = 0;
    box_hi[a] = a < dim ? 0 : 1;
  }
  if (n_marked <= 0) return EB_OK;
  auto floor_to = [block](long long x) { return (x >= 0 ? x / block : -((-x + block - 1) / block)) * block; };
  auto ceil_to = [block](long long x) { return (x >= 0 ? (x + block - 1) / block : -((-x) / block)) * block; };
  int lo[3], hi[3];
  for (int a = 0; a < dim; ++a) {
    long long l = floor_to((long long)bbox_lo[a] - buf), h = ceil_to((long long)bbox_hi[a] + buf);
    const long long lmin = cf_lo[a] ? block : 0, hmax = cf_hi[a] ? (long long)n[a] - block : n[a];
    l = std::max(l, lmin);
    h = std::min(h, hmax);
    if (h - l < block) {  // widened away from the clipped side to one block
      if (l == lmin) h = l + block;
      else l = h - block;
      if (l < lmin || h > hmax) return EB_OK;
    }
    lo[a] = (int)l;
    hi[a] = (int)h;
  }
  for (int a = 0; a < dim; ++a) {
    box_lo[a] = lo[a];
    box_hi[a] = hi[a];
  }
  *has_box = 1;
  return EB_OK;
}
