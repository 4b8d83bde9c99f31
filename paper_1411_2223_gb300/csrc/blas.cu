// CG vector kernels (the start r = b, p = r with |b|^2; p = a r + beta p;
// the scalar steps after the Dslash kernels' reductions)
// and the canonical <-> packed colour-vector conversions.  The update
// xs += alpha p, r -= alpha Ap with |r|^2 runs in the epilogue of the second
// Dslash (MODE_UPDATE of dslash.cuh).  All are bandwidth-bound streaming
// kernels: one thread per site, 16-byte accesses, one right-hand side per
// grid row (blockIdx.y).
#include "sq_device.cuh"
#include "cg_finish.cuh"
#include "sq_kernels.h"

namespace sq {

namespace {

__device__ __forceinline__ bool running(const SlotState *s) { return s->status == SLOT_RUNNING; }

// p = a r + beta p (a complex, 1 except right after a reliable update)
template <int S>
__global__ void __launch_bounds__(256, S == PREC_F64 ? 4 : 8) cg_xpay_kernel(VecArgs a) {
  using R = typename SpinorIO<S>::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  const int St = a.g.stride;
  // p was last written at least two kernels back (r is the predecessor's)
  Vec3<R> p;
  if (i < a.g.vh) p = SpinorIO<S>::load(a.p + r * a.fb, St, i);
  griddep_wait();
  griddep_launch_dependents();
  const SlotState *s = a.slots + r;
  if (i >= a.g.vh || !running(s)) return;
  const R are = (R)s->a_re, aim = (R)s->a_im, beta = (R)s->beta;
  Vec3<R> rv = SpinorIO<S>::load(a.r + r * a.fb, St, i);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R px = fma(are, rv.c[c].x, fma(-aim, rv.c[c].y, beta * p.c[c].x));
    R py = fma(are, rv.c[c].y, fma(aim, rv.c[c].x, beta * p.c[c].y));
    p.c[c].x = px;
    p.c[c].y = py;
  }
  SpinorIO<S>::store(a.p + r * a.fb, St, i, p);
}

// The CG's scalar step after a sloppy Dslash kernel: the kernel's per-warp
// partial sums of each system are added in a fixed order by FINISH_BLOCKS
// blocks (a fixed partition of the partials, so that the FP64 adds are
// spread over as many SMs: GB300 issues about two FP64 adds per clock per
// SM, and one block would spend ~3 us on a 20^3 x 64 lattice's 8000
// partials alone); the block that arrives last (a ticket per system) adds
// the block sums in order and runs finish_alpha (KIND 0: after the D_oe
// kernel, the sum is <p, A p>) or finish_update (KIND 1: after the D_eo
// kernel, the sum is |r|^2).  Systems the Dslash kernel skipped (not
// running) are skipped here too.  Launched with programmatic stream
// serialization, it lets the next Dslash kernel launch -- and prefetch its
// links -- while it adds.
constexpr int FINISH_THREADS = 256;
constexpr int FINISH_BLOCKS = 16;

// Blocks per system for a lattice: at most FINISH_BLOCKS, and no more than
// the groups of 32 warp partials, whose sum slots hold the block sums.
inline int finish_blocks(const Geom &g) { return g.ngroups < FINISH_BLOCKS ? g.ngroups : FINISH_BLOCKS; }

template <int KIND>
__global__ void __launch_bounds__(FINISH_THREADS) cg_finish_kernel(VecArgs a) {
  __shared__ double smem[FINISH_THREADS / 32];
  griddep_wait();
  griddep_launch_dependents();
  const int sys = blockIdx.y, j = blockIdx.x, nb = gridDim.x;
  SlotState *s = a.slots + sys;
  if (s->status != SLOT_RUNNING) return;  // the same in every block of the system
  const int n = a.g.nwchunks;
  double *p = a.partial + (size_t)sys * red_stride(a.g);
  const int per = (n + nb - 1) / nb;
  const int k0 = j * per, k1 = min(n, k0 + per);
  double v = 0.0;
  for (int k = k0 + (int)threadIdx.x; k < k1; k += FINISH_THREADS) v += __ldcg(p + k);
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bs = 0.0;
#pragma unroll
    for (int w = 0; w < FINISH_THREADS / 32; ++w) bs += smem[w];
    p[n + j] = bs;  // the group-sum slots of this reduction instance
    unsigned *ticket = a.counter + (size_t)sys * ticket_stride(a.g);
    if (atom_add_acq_rel(ticket, 1u) == (unsigned)(nb - 1)) {
      double sum = 0.0;
      for (int b = 0; b < nb; ++b) sum += __ldcg(p + n + b);
      *ticket = 0;
      if (KIND == 0) finish_alpha(s, sum);
      else finish_update(s, sum, a.checkpoint);
    }
  }
}

// Start of the systems in SLOT_INIT: r = b (sloppy), p = r, x64 = 0; or with
// an initial guess p = 0 and a pending FP64 residual.  Partial |b|^2; last
// block: finish_init.  Slots already iterating are left alone, so systems
// can join a running batch.
template <int S>
__global__ void __launch_bounds__(256, S == PREC_F64 ? 4 : 8) cg_init_kernel(VecArgs a, int guess) {
  griddep_wait();
  griddep_launch_dependents();
  using R = typename SpinorIO<S>::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  const int St = a.g.stride;
  SlotState *s = a.slots + r;
  if (s->status != SLOT_INIT) return;  // the same for every block of the row
  double val[1] = {0.0};
  if (i < a.g.vh) {
    Vec3<double> b = SpinorIO<PREC_F64>::load(a.b64 + r * a.f64_fb, St, i);
    double n2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) n2 = fma(b.c[c].x, b.c[c].x, fma(b.c[c].y, b.c[c].y, n2));
    val[0] = n2;
    {
      constexpr int XP = (S == PREC_F64) ? PREC_F64 : PREC_F32;
      Vec3<typename SpinorIO<XP>::R> z;
      zero(z);
      SpinorIO<XP>::store(a.xs + r * a.xs_fb, St, i, z);
    }
    if (guess) {
      Vec3<R> z;
      zero(z);
      SpinorIO<S>::store(a.p + r * a.fb, St, i, z);
    } else {
      Vec3<R> rv = convert<R>(b);
      SpinorIO<S>::store(a.r + r * a.fb, St, i, rv);
      SpinorIO<S>::store(a.p + r * a.fb, St, i, rv);
      Vec3<double> z;
      zero(z);
      SpinorIO<PREC_F64>::store(a.x64 + r * a.f64_fb, St, i, z);
    }
  }
  double *const inst[1] = {a.partial + (size_t)r * red_stride(a.g)};
  double b2[1];
  unsigned *tickets = a.counter + (size_t)r * ticket_stride(a.g);
  if (warp_tree_reduce<1>(val, 1, inst, a.g, i, tickets, b2) && (threadIdx.x & 31) == 0) {
    finish_init(s, b2[0]);
    if (guess && s->status == SLOT_RUNNING) {
      s->ru_pending = 1;
      s->status = SLOT_WAIT;
    }
  }
}

// canonical [i][colour] complex128 -> packed precision P (nrhs fields)
template <int P>
__global__ void pack_kernel(Geom g, const double2 *canon, size_t canon_fe, char *out,
                            size_t out_fb) {
  using R = typename SpinorIO<P>::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= g.vh) return;
  const double2 *c = canon + r * canon_fe + (size_t)3 * i;
  Vec3<double> v;
#pragma unroll
  for (int k = 0; k < 3; ++k) v.c[k] = c[k];
  SpinorIO<P>::store(out + r * out_fb, g.stride, i, convert<R>(v));
}

template <int P>
__global__ void unpack_kernel(Geom g, const char *in, size_t in_fb, double2 *canon,
                              size_t canon_fe) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= g.vh) return;
  auto v = SpinorIO<P>::load(in + r * in_fb, g.stride, i);
  double2 *c = canon + r * canon_fe + (size_t)3 * i;
#pragma unroll
  for (int k = 0; k < 3; ++k) c[k] = make_double2((double)v.c[k].x, (double)v.c[k].y);
}

// x64 (packed FP64) <-> canonical for the solution / source of a solve
template <int P>
__global__ void convert_kernel(Geom g, const char *in, size_t in_fb, char *out, size_t out_fb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= g.vh) return;
  auto v = SpinorIO<PREC_F64>::load(in + r * in_fb, g.stride, i);
  SpinorIO<P>::store(out + r * out_fb, g.stride, i, convert<typename SpinorIO<P>::R>(v));
}

inline dim3 grid_for(const Geom &g, int block, int nrhs) {
  return dim3((g.vh + block - 1) / block, nrhs);
}

}  // namespace

int launch_cg_xpay(int prec, const VecArgs &a, cudaStream_t st) {
  if (a.g.vh <= 0) return 0;
  dim3 grid = grid_for(a.g, 256, a.nrhs);
  switch (prec) {
    case PREC_F64: if (launch_pdl(cg_xpay_kernel<PREC_F64>, grid, dim3(256), 0, st, a)) return -1; break;
    case PREC_F32: if (launch_pdl(cg_xpay_kernel<PREC_F32>, grid, dim3(256), 0, st, a)) return -1; break;
    case PREC_I16: if (launch_pdl(cg_xpay_kernel<PREC_I16>, grid, dim3(256), 0, st, a)) return -1; break;
    default: return -1;
  }
  return 0;
}

int launch_cg_finish(int kind, const VecArgs &a, cudaStream_t st) {
  if (a.g.vh <= 0) return 0;
  const dim3 grid(finish_blocks(a.g), a.nrhs), block(FINISH_THREADS);
  cudaError_t e = (kind == 0) ? launch_pdl(cg_finish_kernel<0>, grid, block, 0, st, a)
                              : launch_pdl(cg_finish_kernel<1>, grid, block, 0, st, a);
  return e == cudaSuccess ? 0 : -1;
}

int launch_cg_init(int prec, const VecArgs &a, int guess, cudaStream_t st) {
  if (a.g.vh <= 0) return 0;
  dim3 grid = grid_for(a.g, 256, a.nrhs);
  switch (prec) {
    case PREC_F64: if (launch_pdl(cg_init_kernel<PREC_F64>, grid, dim3(256), 0, st, a, guess)) return -1; break;
    case PREC_F32: if (launch_pdl(cg_init_kernel<PREC_F32>, grid, dim3(256), 0, st, a, guess)) return -1; break;
    case PREC_I16: if (launch_pdl(cg_init_kernel<PREC_I16>, grid, dim3(256), 0, st, a, guess)) return -1; break;
    default: return -1;
  }
  return 0;
}

int launch_pack(int prec, const Geom &g, const double *canon, size_t canon_elems, void *out,
                size_t out_fb, int nrhs, cudaStream_t st) {
  if (g.vh <= 0) return 0;
  dim3 grid = grid_for(g, 256, nrhs);
  const double2 *c = reinterpret_cast<const double2 *>(canon);
  char *o = static_cast<char *>(out);
  switch (prec) {
    case PREC_F64: pack_kernel<PREC_F64><<<grid, 256, 0, st>>>(g, c, canon_elems, o, out_fb); break;
    case PREC_F32: pack_kernel<PREC_F32><<<grid, 256, 0, st>>>(g, c, canon_elems, o, out_fb); break;
    case PREC_I16: pack_kernel<PREC_I16><<<grid, 256, 0, st>>>(g, c, canon_elems, o, out_fb); break;
    default: return -1;
  }
  return 0;
}

int launch_unpack(int prec, const Geom &g, const void *in, size_t in_fb, double *canon,
                  size_t canon_elems, int nrhs, cudaStream_t st) {
  if (g.vh <= 0) return 0;
  dim3 grid = grid_for(g, 256, nrhs);
  double2 *c = reinterpret_cast<double2 *>(canon);
  const char *p = static_cast<const char *>(in);
  switch (prec) {
    case PREC_F64: unpack_kernel<PREC_F64><<<grid, 256, 0, st>>>(g, p, in_fb, c, canon_elems); break;
    case PREC_F32: unpack_kernel<PREC_F32><<<grid, 256, 0, st>>>(g, p, in_fb, c, canon_elems); break;
    case PREC_I16: unpack_kernel<PREC_I16><<<grid, 256, 0, st>>>(g, p, in_fb, c, canon_elems); break;
    default: return -1;
  }
  return 0;
}

int launch_convert_from_f64(int prec, const Geom &g, const void *in, size_t in_fb, void *out,
                            size_t out_fb, int nrhs, cudaStream_t st) {
  if (g.vh <= 0) return 0;
  dim3 grid = grid_for(g, 256, nrhs);
  const char *p = static_cast<const char *>(in);
  char *o = static_cast<char *>(out);
  switch (prec) {
    case PREC_F64: convert_kernel<PREC_F64><<<grid, 256, 0, st>>>(g, p, in_fb, o, out_fb); break;
    case PREC_F32: convert_kernel<PREC_F32><<<grid, 256, 0, st>>>(g, p, in_fb, o, out_fb); break;
    case PREC_I16: convert_kernel<PREC_I16><<<grid, 256, 0, st>>>(g, p, in_fb, o, out_fb); break;
    default: return -1;
  }
  return 0;
}

}  // namespace sq
