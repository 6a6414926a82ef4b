// The nested SRHT transform (Sec. 2.2): Z = H D P [X Y; 0] over N' = 2^n
// padded rows, H the normalised Sylvester Walsh-Hadamard matrix.
//
// H_{N'} factors over groups of index bits: a pass that owns bits
// [s, s + b) runs the 2^b-point transform on every set of rows that differ
// only in those bits.  Each CTA stages one such set (2^b rows, rows 2^s
// apart) for a slab of TC adjacent columns in shared memory, runs the b
// butterfly levels there and writes the slab back.  The first pass fuses
// the signed row gather (D P), the last pass fuses the 1/sqrt(N') scale and
// the scatter of the rows of I_K (to their position in pi order) and of
// I-hat (scaled by sqrt(N'/r), column-major for the QR).  Y is column d.
#include "common.cuh"
#include "internal.hpp"

namespace spcg {

struct FwhtArgs {
  // source of the first pass
  const double* X;
  int64_t ldx;
  const double* Y;
  int64_t N;
  const uint32_t* gather;
  // work buffer
  double* W;
  int64_t ldw;
  int C;             // d + 1 columns (Y last)
  int d;
  int nbits;         // log2 N'
  int shift;         // low bit of this pass
  int first, last;
  int ncoltiles;
  // scatter of the last pass
  const int32_t* dest;
  const int32_t* hdest;
  double* AK;
  int64_t ldak;
  double* bK;
  double* Ahat;      // column-major, ld = r
  int64_t r;
  double scale;      // 1/sqrt(N')
  double hat_scale;  // sqrt(N'/r)
};

template <int LOGL>
struct FwhtShape {
  static constexpr int L = 1 << LOGL;
  static constexpr int TC = (L <= 1024) ? 16 : (L == 2048 ? 8 : 4);
  static constexpr int THREADS = 512;
  static constexpr size_t SMEM = (size_t)L * TC * sizeof(double) + (size_t)L * 3 * sizeof(int32_t);
};

template <int LOGL>
__global__ void __launch_bounds__(512) k_fwht_pass(const FwhtArgs a) {
  using S = FwhtShape<LOGL>;
  constexpr int L = S::L, TC = S::TC, NT = S::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* tile = reinterpret_cast<double*>(smem_raw);
  int32_t* gmap = reinterpret_cast<int32_t*>(tile + (size_t)L * TC);  // gather (first pass)
  int32_t* dmap = gmap + L;                                             // dest (last pass)
  int32_t* hmap = dmap + L;                                             // hdest (last pass)

  const int64_t blk = blockIdx.x;
  const int ct = (int)(blk % a.ncoltiles);
  const int64_t base = blk / a.ncoltiles;
  const int c0 = ct * TC;
  const int64_t low = base & ((int64_t(1) << a.shift) - 1);
  const int64_t high = base >> a.shift;
  // global row of tile row t
  auto grow = [&](int t) -> int64_t {
    return low | ((int64_t)t << a.shift) | (high << (a.shift + LOGL));
  };

  const int tid = threadIdx.x;
  if (a.first) {
    for (int t = tid; t < L; t += NT) gmap[t] = (int32_t)a.gather[grow(t)];
  }
  if (a.last) {
    for (int t = tid; t < L; t += NT) {
      const int64_t j = grow(t);
      dmap[t] = a.dest[j];
      hmap[t] = a.hdest[j];
    }
  }
  __syncthreads();

  // load
  for (int e = tid; e < L * TC; e += NT) {
    const int t = e / TC, c = e % TC;
    const int col = c0 + c;
    double v = 0.0;
    if (col < a.C) {
      if (a.first) {
        const uint32_t gm = (uint32_t)gmap[t];
        const int64_t src = (int64_t)(gm & 0x7FFFFFFFu);
        if (src < a.N) {
          v = (col < a.d) ? a.X[src * a.ldx + col] : a.Y[src];
          if (gm & 0x80000000u) v = -v;
        }
      } else {
        v = a.W[grow(t) * a.ldw + col];
      }
    }
    tile[e] = v;
  }
  __syncthreads();

  // radix-2 butterflies over the LOGL bits of the tile row index
#pragma unroll 1
  for (int h = 1; h < L; h <<= 1) {
    for (int q = tid; q < (L / 2) * TC; q += NT) {
      const int c = q % TC, pr = q / TC;
      const int t = (pr / h) * 2 * h + (pr % h);
      const double x = tile[t * TC + c], y = tile[(t + h) * TC + c];
      tile[t * TC + c] = x + y;
      tile[(t + h) * TC + c] = x - y;
    }
    __syncthreads();
  }

  // store
  for (int e = tid; e < L * TC; e += NT) {
    const int t = e / TC, c = e % TC;
    const int col = c0 + c;
    if (col >= a.C) continue;
    double v = tile[e];
    if (!a.last) {
      a.W[grow(t) * a.ldw + col] = v;
    } else {
      v *= a.scale;
      const int32_t dst = dmap[t];
      if (dst >= 0) {
        if (col < a.d) a.AK[(int64_t)dst * a.ldak + col] = v;
        else a.bK[dst] = v;
      }
      const int32_t hd = hmap[t];
      if (hd >= 0 && col < a.d) a.Ahat[(int64_t)col * a.r + hd] = v * a.hat_scale;
    }
  }
}

template <int LOGL>
static spcg_status launch_one(const FwhtArgs& a, int64_t nbases, cudaStream_t st) {
  using S = FwhtShape<LOGL>;
  FwhtArgs b = a;
  b.ncoltiles = (a.C + S::TC - 1) / S::TC;
  const size_t smem = S::SMEM;
  SPCG_CK(cudaFuncSetAttribute(k_fwht_pass<LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  const int64_t nblk = nbases * b.ncoltiles;
  k_fwht_pass<LOGL><<<(unsigned)nblk, S::THREADS, smem, st>>>(b);
  SPCG_CK(cudaGetLastError());
  return SPCG_OK;
}

static spcg_status launch_logl(int logl, const FwhtArgs& a, int64_t nbases, cudaStream_t st) {
  switch (logl) {
    case 1: return launch_one<1>(a, nbases, st);
    case 2: return launch_one<2>(a, nbases, st);
    case 3: return launch_one<3>(a, nbases, st);
    case 4: return launch_one<4>(a, nbases, st);
    case 5: return launch_one<5>(a, nbases, st);
    case 6: return launch_one<6>(a, nbases, st);
    case 7: return launch_one<7>(a, nbases, st);
    case 8: return launch_one<8>(a, nbases, st);
    case 9: return launch_one<9>(a, nbases, st);
    case 10: return launch_one<10>(a, nbases, st);
    case 11: return launch_one<11>(a, nbases, st);
    case 12: return launch_one<12>(a, nbases, st);
    default: return SPCG_E_INVALID_ARG;
  }
}

// Split n index bits into passes of at most 12 bits, as even as possible.
int fwht_pass_plan(int n, int* logl) {
  const int passes = (n + 11) / 12;
  for (int p = 0; p < passes; ++p) logl[p] = n / passes + (p < n % passes ? 1 : 0);
  return passes;
}

spcg_status launch_transform(spcg_ctx* c) {
  Sketch& s = c->sk;
  int logl[8];
  const int passes = fwht_pass_plan(s.nbits, logl);
  FwhtArgs a{};
  a.X = c->X;
  a.ldx = c->ldx;
  a.Y = c->Y;
  a.N = c->N;
  a.gather = s.gather;
  a.W = s.work;
  a.ldw = s.ldw;
  a.C = c->d + 1;
  a.d = c->d;
  a.nbits = s.nbits;
  a.dest = s.dest;
  a.hdest = s.hdest;
  a.AK = s.AK;
  a.ldak = s.ldak;
  a.bK = s.bK;
  a.Ahat = s.Ahat;
  a.r = s.sched.r;
  a.scale = 1.0 / sqrt((double)s.n_pad);
  a.hat_scale = sqrt((double)s.n_pad / (double)s.sched.r);
  int shift = 0;
  for (int p = 0; p < passes; ++p) {
    a.shift = shift;
    a.first = (p == 0);
    a.last = (p == passes - 1);
    const int64_t nbases = s.n_pad >> logl[p];
    SPCG_TRY(launch_logl(logl[p], a, nbases, c->stream));
    c->n_launch += 1;
    shift += logl[p];
  }
  return SPCG_OK;
}

}  // namespace spcg
