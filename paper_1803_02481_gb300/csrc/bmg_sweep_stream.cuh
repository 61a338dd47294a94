// Streaming red-black Gauss-Seidel sweep of a 5-point level (smoothing of
// Algorithm 1), for large levels.
//
// A thread block owns a strip of 2*NT - 2 columns and R rows.  Thread t owns
// the column pair (a, a+1), a = cs + 2t, where cs is the strip's first column
// minus one; the outermost two columns are a halo whose red values are
// recomputed here (the neighbouring strip computes the same values).  Rows
// stream through a ring of NSLOT shared-memory rows filled by cp.async three
// rows ahead.  In the step for row j, every thread relaxes the red point of
// row j in its pair and then the black point of row j-1 in the same column
// (its other neighbours are red points of rows j-2..j, all final by then),
// and row j-1 is written out.  The old iterate is read from one buffer and
// the new one written to another, so strips never see each other's new
// values.  Per-point arithmetic is gs_apply, shared with every other kernel.
#pragma once

#include "bmg_internal.h"

namespace bmg {

namespace stream_detail {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Asynchronous copy of one element (4 or 8 bytes) into shared memory; when
// `valid` is false nothing is read and the destination is zero-filled.
template <typename T>
__device__ __forceinline__ void cp_elem(T* dst, const T* src, bool valid) {
  const unsigned d = smem_addr(dst);
  const int n = valid ? int(sizeof(T)) : 0;
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n));
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }

template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

}  // namespace stream_detail

template <typename T, int NT, int R>
struct StreamRB {
  static constexpr int SW = 2 * NT + 2;   // shared columns q: plane column cs-1+q
  static constexpr int NSLOT = 7;         // rows j-2 .. j+4
  static constexpr int OWN = 2 * NT - 2;  // columns written per strip
  static constexpr int HALF = NT + 1;     // columns of one parity
  // One ring row, split by column parity so that a warp's accesses are
  // contiguous: column q lives at index q >> 1 of the array of parity q & 1.
  struct Arr {
    T v[2][HALF];
  };
  struct Row {
    Arr x, ic, w, s, b;
  };
};

// Red-black sweep of one strip: rows [r0, r0 + R) of columns [c0, c0 + OWN).
template <typename T, int NT, int R>
__device__ __forceinline__ void sweep_rb_strip(const LevelV<T>& L, const T* __restrict__ xin,
                                               T* __restrict__ xout, bool reverse, int c0,
                                               int r0) {
  using namespace stream_detail;
  using S = StreamRB<T, NT, R>;
  constexpr int SW = S::SW, NSLOT = S::NSLOT;
  extern __shared__ __align__(16) unsigned char stream_smem[];
  typename S::Row* ring = reinterpret_cast<typename S::Row*>(stream_smem);
  const int nx = L.nx, ny = L.ny, p = L.pitch;
  const int cs = c0 - 1;          // first red column of the strip
  const int rbase = r0 - 2;       // first row loaded
  const int rlast = r0 + R + 1;   // last row loaded
  const int t = threadIdx.x;
  const int first_parity = reverse ? 1 : 0;   // (i + j + first_parity) even: first colour

  auto load_row = [&](int j) {
    typename S::Row& rw = ring[(j - rbase) % NSLOT];
    const bool rowok = j >= 0 && j <= ny + 1;
    for (int q = t; q < SW; q += NT) {
      const int i = cs - 1 + q;
      const bool ok = rowok && i >= 0 && i <= nx + 1;
      const int o = ok ? j * p + i : 0;
      const int par = q & 1, k = q >> 1;
      cp_elem<T>(&rw.x.v[par][k], xin + o, ok);
      cp_elem<T>(&rw.ic.v[par][k], L.iC + o, ok);
      cp_elem<T>(&rw.w.v[par][k], L.W + o, ok);
      cp_elem<T>(&rw.s.v[par][k], L.S + o, ok);
      cp_elem<T>(&rw.b.v[par][k], L.b + o, ok);
    }
    cp_commit();
  };

  // Relax the point of column q in ring row j (neighbours in rows j-1, j+1).
  auto relax = [&](int j, int q) {
    typename S::Row& rc = ring[(j - rbase) % NSLOT];
    const typename S::Row& rs = ring[(j - 1 - rbase) % NSLOT];
    const typename S::Row& rn = ring[(j + 1 - rbase) % NSLOT];
    const int par = q & 1, k = q >> 1;
    const int opar = par ^ 1;
    // q - 1 and q + 1 have the other parity, at indices (q-1)>>1, (q+1)>>1
    const int km = (q - 1) >> 1, kp = (q + 1) >> 1;
    GsCoef<T, false> c;
    c.b = rc.b.v[par][k];
    c.ic = rc.ic.v[par][k];
    c.w = rc.w.v[par][k];
    c.e = rc.w.v[opar][kp];
    c.s = rc.s.v[par][k];
    c.n = rn.s.v[par][k];
    rc.x.v[par][k] = gs_apply<T, false>(c, [&](int dx, int dy) {
      return dy == 0 ? rc.x.v[opar][dx < 0 ? km : kp] : (dy < 0 ? rs.x.v[par][k] : rn.x.v[par][k]);
    });
  };

  // rows rbase .. rbase + 4 in flight before the first step
#pragma unroll
  for (int k = 0; k < 5; ++k) load_row(rbase + k);

  const int qa = 1 + 2 * t;       // shared column of the thread's first column
  for (int jr = r0 - 1; jr <= r0 + R; ++jr) {
    // rows up to jr + 1 have landed (jr + 2 and jr + 3 may be in flight)
    cp_wait<2>();
    __syncthreads();
    if (jr + 4 <= rlast) load_row(jr + 4);
    else cp_commit();             // keep the group count uniform
    // first colour at row jr, in the column of the pair with the right parity
    const int ia = cs + 2 * t;
    const int q = ((ia + jr + first_parity) & 1) ? qa + 1 : qa;
    const int i = cs - 1 + q;
    if (jr >= 1 && jr <= ny && i >= 1 && i <= nx) relax(jr, q);
    __syncthreads();
    // second colour at row jb = jr - 1, same column
    const int jb = jr - 1;
    if (jb >= r0) {
      const bool own = q >= 2 && q <= SW - 3;   // not a halo column
      if (own && jb >= 1 && jb <= ny && i >= 1 && i <= nx) relax(jb, q);
      // row jb is final: write the thread's own columns of it
      if (jb >= 1 && jb <= ny) {
        const typename S::Row& rc = ring[(jb - rbase) % NSLOT];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int qq = qa + k;
          const int ii = cs - 1 + qq;
          if (qq >= 2 && qq <= SW - 3 && ii >= 1 && ii <= nx)
            xout[jb * p + ii] = rc.x.v[qq & 1][qq >> 1];
        }
      }
    }
  }
  cp_wait<0>();
}

template <typename T, int NT, int R>
__global__ void __launch_bounds__(NT) k_sweep_rb_stream(LevelV<T> L, const T* __restrict__ xin,
                                                        T* __restrict__ xout, int reverse) {
  const int c0 = 1 + blockIdx.x * StreamRB<T, NT, R>::OWN;
  const int r0 = 1 + blockIdx.y * R;
  sweep_rb_strip<T, NT, R>(L, xin, xout, reverse != 0, c0, r0);
}

}  // namespace bmg
