// Batched Stockham FFT core shared by the FP32 stress passes and the FP64
// kernel-spectrum build.
//
// Layout convention: a tile of W independent lines of length P lives in shared
// memory interleaved, element n of line w at buf[n * LD + w].  Consecutive
// threads take consecutive lines w, so every shared-memory access of a pass is
// a contiguous run of W complex values (no transposes between passes).
//
// One pass of radix R on length-P transforms with current span Ns (the
// Stockham autosort formulation, Govindaraju et al., SC'08):
//   butterfly j in [0, P/R): inputs n = j + r P/R (r = 0..R-1), twiddled by
//   exp(-+2 pi i (j mod Ns) r / (Ns R)), an R-point DFT in registers, outputs
//   written to n' = (j / Ns) Ns R + (j mod Ns) + r Ns.
// All reads of a pass happen before the barrier, all writes after it, so one
// buffer suffices.  Forward transforms are unnormalised, exp(-2 pi i nk / P);
// inverse ones use exp(+2 pi i nk / P), also unnormalised.
//
// Two zero-aware variants serve the zero-padded convolution:
//   ZIN : only the first P/2 inputs are non-zero (the first pass skips the rest);
//   HOUT: only the first P/2 outputs are wanted (the last pass stores only them).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dds {

template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <typename C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

// a * w (INV=false) or a * conj(w) (INV=true)
template <bool INV>
__device__ __forceinline__ float2 cmul_tw(float2 a, float2 w) {
  if (INV) return make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
  return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
template <bool INV>
__device__ __forceinline__ double2 cmul_tw(double2 a, double2 w) {
  if (INV) return make_double2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
  return make_double2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}

// cos(2 pi q / 32), q = 0..31 (decimal expansions of the constants).
__device__ __forceinline__ constexpr double c32(int q) {
  constexpr double t[9] = {1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
                           0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173,
                           0.19509032201612826785, 0.0};
  q &= 31;
  return q <= 8 ? t[q] : q <= 16 ? -t[16 - q] : q <= 24 ? -t[q - 16] : t[32 - q];
}
__device__ __forceinline__ constexpr double s32(int q) { return c32(q - 8); }   // sin(a) = cos(a - pi/2)

// multiply by exp(-+2 pi i k / n) for compile-time k < n <= 32, special-casing
// the quarter turns so that no multiply by 0 or 1 is issued.
template <bool INV, typename C>
__device__ __forceinline__ C rot_const(C a, int k, int n) {
  const int q = (32 / n) * k;     // angle index in 32nds of a turn
  if (q == 0) return a;
  if (q == 8) { C r; r.x = INV ? -a.y : a.y; r.y = INV ? a.x : -a.x; return r; }    // * (-+ i)
  if (q == 16) { C r; r.x = -a.x; r.y = -a.y; return r; }
  if (q == 24) { C r; r.x = INV ? a.y : -a.y; r.y = INV ? -a.x : a.x; return r; }   // * (+- i)
  using T = decltype(a.x);
  const T c = (T)c32(q);
  const T s = INV ? (T)s32(q) : -(T)s32(q);
  C r;
  r.x = a.x * c - a.y * s;
  r.y = a.x * s + a.y * c;
  return r;
}

// In-register R-point DFT (R = 2 .. 32): radix-2 decimation in time written
// as a template recursion, so every register index is a compile-time constant.
template <int R, bool INV, typename C>
struct DftReg {
  static __device__ __forceinline__ void run(C* v) {
    C ev[R / 2], od[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      ev[i] = v[2 * i];
      od[i] = v[2 * i + 1];
    }
    DftReg<R / 2, INV, C>::run(ev);
    DftReg<R / 2, INV, C>::run(od);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      const C w = rot_const<INV>(od[k], k, R);
      v[k] = cadd(ev[k], w);
      v[k + R / 2] = csub(ev[k], w);
    }
  }
};
template <bool INV, typename C>
struct DftReg<1, INV, C> {
  static __device__ __forceinline__ void run(C*) {}
};

template <int R, bool INV, typename C>
__device__ __forceinline__ void dft_reg(C* v) {
  DftReg<R, INV, C>::run(v);
}

// Radix plans: product of the entries = P, applied first to last.
template <int P> struct Plan;
template <> struct Plan<16>   { static constexpr int n = 1, r0 = 16, r1 = 1, r2 = 1; };
template <> struct Plan<32>   { static constexpr int n = 2, r0 = 8,  r1 = 4, r2 = 1; };
template <> struct Plan<64>   { static constexpr int n = 2, r0 = 8,  r1 = 8, r2 = 1; };
template <> struct Plan<128>  { static constexpr int n = 2, r0 = 16, r1 = 8, r2 = 1; };
template <> struct Plan<256>  { static constexpr int n = 2, r0 = 16, r1 = 16, r2 = 1; };
template <> struct Plan<512>  { static constexpr int n = 2, r0 = 16, r1 = 32, r2 = 1; };
template <> struct Plan<1024> { static constexpr int n = 2, r0 = 32, r1 = 32, r2 = 1; };

// Asynchronous global -> shared copies (cp.async): every thread issues all of
// its copies before waiting, so a whole tile is in flight at once.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N committed groups of this thread are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Twiddle tables: for every power of two P in [16, 2048] the values
// exp(-2 pi i k / P), k = 0..P-1, stored back to back starting at offset P - 16.
__host__ __device__ constexpr int tw_offset(int P) { return P - 16; }
constexpr int TW_TOTAL = 4096 - 16;

template <typename C>
__device__ __forceinline__ C tw_load(const C* tw, int idx) {
  return __ldg(tw + idx);
}

// Address of element n of line w in a tile of W lines.  With PADB > 0 every block
// of PADB rows is shifted by W elements: the first pass writes rows R0 apart, and
// without the shift the W-element groups of the butterflies a warp handles at once
// land on the same shared-memory banks whenever the tile is narrower than 16 lines.
template <int LD, int PADB, int W>
__device__ __forceinline__ int tidx(int n, int w) {
  return n * LD + w + (PADB > 0 ? (n / PADB) * W : 0);
}
template <int P, int LD, int PADB, int W>
__host__ __device__ constexpr int tile_elems() {
  return P * LD + (PADB > 0 ? (P / PADB) * W : 0);
}

// One Stockham pass over the tile (see file comment).
template <int P, int R, int NS, int W, int LD, int PADB, int NT, bool INV, bool ZIN, bool HOUT, typename C>
__device__ __forceinline__ void stockham_pass(C* buf, const C* twP, int tid) {
  constexpr int NB = (P / R) * W;
  constexpr int PER = (NB + NT - 1) / NT;
  C v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int bi = tid + q * NT;
    if ((NB % NT) == 0 || bi < NB) {
      const int w = bi % W, j = bi / W;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (ZIN && r >= R / 2) v[q][r] = czero<C>();
        else v[q][r] = buf[tidx<LD, PADB, W>(j + r * (P / R), w)];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int bi = tid + q * NT;
    if ((NB % NT) == 0 || bi < NB) {
      const int w = bi % W, j = bi / W;
      const int jm = j % NS;
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const C t = tw_load(twP, jm * r * (P / (NS * R)));
          v[q][r] = cmul_tw<INV>(v[q][r], t);
        }
      }
      dft_reg<R, INV>(v[q]);
      const int base = (j / NS) * NS * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!HOUT || r < R / 2) buf[tidx<LD, PADB, W>(base + r * NS, w)] = v[q][r];
      }
    }
  }
  __syncthreads();
}

// Full length-P FFT of the W lines of a tile.  twP points at the P-table.
// PADB: 0 for a plain [P][LD] tile, or Plan<P>::r0 for the shifted layout (tidx).
template <int P, int W, int LD, int NT, bool INV, bool ZIN, bool HOUT, int PADB = 0, typename C>
__device__ __forceinline__ void fft_tile(C* buf, const C* twP, int tid) {
  using PL = Plan<P>;
  stockham_pass<P, PL::r0, 1, W, LD, PADB, NT, INV, ZIN, (PL::n == 1) && HOUT>(buf, twP, tid);
  if constexpr (PL::n >= 2)
    stockham_pass<P, PL::r1, PL::r0, W, LD, PADB, NT, INV, false, (PL::n == 2) && HOUT>(buf, twP, tid);
  if constexpr (PL::n >= 3)
    stockham_pass<P, PL::r2, PL::r0 * PL::r1, W, LD, PADB, NT, INV, false, HOUT>(buf, twP, tid);
}

// Variant with a runtime number of interleaved lines L <= LMAX (row pitch L):
// lets one pass transform several fields (or components) of a tile together.
template <int P, int R, int NS, int LMAX, int NT, bool INV, bool ZIN, bool HOUT, typename C>
__device__ __forceinline__ void stockham_pass_rt(C* buf, int L, const C* twP, int tid) {
  constexpr int PER = ((P / R) * LMAX + NT - 1) / NT;
  const int NB = (P / R) * L;
  C v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int bi = tid + q * NT;
    if (bi < NB) {
      const int j = bi / L, w = bi - j * L;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (ZIN && r >= R / 2) v[q][r] = czero<C>();
        else v[q][r] = buf[(j + r * (P / R)) * L + w];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int bi = tid + q * NT;
    if (bi < NB) {
      const int j = bi / L, w = bi - j * L;
      const int jm = j % NS;
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[q][r] = cmul_tw<INV>(v[q][r], tw_load(twP, jm * r * (P / (NS * R))));
      }
      dft_reg<R, INV>(v[q]);
      const int base = (j / NS) * NS * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!HOUT || r < R / 2) buf[(base + r * NS) * L + w] = v[q][r];
      }
    }
  }
  __syncthreads();
}

template <int P, int LMAX, int NT, bool INV, bool ZIN, bool HOUT, typename C>
__device__ __forceinline__ void fft_tile_rt(C* buf, int L, const C* twP, int tid) {
  using PL = Plan<P>;
  stockham_pass_rt<P, PL::r0, 1, LMAX, NT, INV, ZIN, (PL::n == 1) && HOUT>(buf, L, twP, tid);
  if constexpr (PL::n >= 2)
    stockham_pass_rt<P, PL::r1, PL::r0, LMAX, NT, INV, false, (PL::n == 2) && HOUT>(buf, L, twP, tid);
  if constexpr (PL::n >= 3)
    stockham_pass_rt<P, PL::r2, PL::r0 * PL::r1, LMAX, NT, INV, false, HOUT>(buf, L, twP, tid);
}

}  // namespace dds
