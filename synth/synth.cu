// GPU twins of the seeded input generators in synth/__init__.py, for inputs
// too large to build on the host (n = 10^9).  Input generation only: nothing
// here computes a step of the semisort method.  Integer generators reproduce
// the CPU twins bit for bit; the floating-point ones (Zipf, exponential,
// Gaussian mixture) follow the same formulas with CUDA's math library.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStreamMul = 0xD1B54A32D192ED03ull;

__host__ __device__ inline uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t stream_base(uint64_t seed, uint64_t stream) { return mix(seed ^ (stream * kStreamMul)); }
__device__ inline uint64_t rand64(uint64_t base, uint64_t ctr) { return mix(base + (ctr + 1) * kGolden); }
__device__ inline double unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

#define GRID_STRIDE(i, count) \
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (count); i += (uint64_t)gridDim.x * blockDim.x)

__global__ void k_iota(uint64_t* out, uint64_t count, uint64_t start) {
  GRID_STRIDE(i, count) out[i] = start + i;
}

__global__ void k_iota32(uint32_t* out, uint64_t count, uint64_t start) {
  GRID_STRIDE(i, count) out[i] = (uint32_t)(start + i);
}

__global__ void k_uniform_mod(uint64_t* out, uint64_t count, uint64_t start, uint64_t seed, uint64_t mu) {
  GRID_STRIDE(i, count) out[i] = mix(seed + (start + i + 1) * kGolden) % mu;
}

struct Feistel {
  uint32_t half;
  uint64_t mask;
  uint64_t rk[4];
};

__device__ inline uint64_t feistel_enc(const Feistel& f, uint64_t x) {
  uint64_t l = x >> f.half, r = x & f.mask;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint64_t t = mix(r ^ f.rk[k]) & f.mask;
    const uint64_t nl = r;
    r = l ^ t;
    l = nl;
  }
  return (l << f.half) | r;
}

__global__ void k_uniform_exact(uint64_t* out, uint64_t count, uint64_t start, uint64_t n, uint64_t mu,
                                Feistel f, uint64_t key_c) {
  GRID_STRIDE(i, count) {
    uint64_t y = feistel_enc(f, start + i);
    while (y >= n) y = feistel_enc(f, y);
    out[i] = mix(y % mu + key_c);
  }
}

// Rejection-inversion for Zipf (Hormann and Derflinger, ACM TOMACS 1996).
// The helpers, constants and acceptance test follow the shape of the Apache
// Commons RNG RejectionInversionZipfSampler (Apache-2.0), a widely used
// statement of the same published method; this is the GPU twin of the numpy
// sampler in synth/__init__.py.
struct ZipfP {
  double s, hx1, hn, sq;
  uint64_t N;
};
__device__ inline double h1(double x) { return fabs(x) < 1e-8 ? 1.0 - x * (0.5 - x * (1.0 / 3.0 - 0.25 * x)) : log1p(x) / x; }
__device__ inline double h2(double x) {
  return fabs(x) < 1e-8 ? 1.0 + x * 0.5 * (1.0 + x * (1.0 / 3.0) * (1.0 + 0.25 * x)) : expm1(x) / x;
}
__device__ inline double zH(const ZipfP& z, double x) {
  const double lx = log(x);
  return h2((1.0 - z.s) * lx) * lx;
}
__device__ inline double zHinv(const ZipfP& z, double x) {
  double t = x * (1.0 - z.s);
  if (t < -1.0) t = -1.0;
  return exp(h1(t) * x);
}
__device__ inline double zh(const ZipfP& z, double x) { return exp(-z.s * log(x)); }

__global__ void k_zipf(uint64_t* out, uint64_t count, uint64_t start, uint64_t seed, ZipfP z, uint64_t key_c,
                       int ranks_only) {
  GRID_STRIDE(i, count) {
    const uint64_t idx = start + i;
    uint64_t k = 1;
    for (uint32_t a = 0; a < 4096; ++a) {
      const uint64_t base = stream_base(seed, 0x21FF + (a >> 6));
      const double u = unit(rand64(base, (idx << 6) | (a & 63)));
      const double v = z.hn + u * (z.hx1 - z.hn);
      const double x = zHinv(z, v);
      double kd = floor(x + 0.5);
      kd = kd < 1.0 ? 1.0 : (kd > (double)z.N ? (double)z.N : kd);
      if (kd - x <= z.sq || v >= zH(z, kd + 0.5) - zh(z, kd)) {
        k = (uint64_t)kd;
        break;
      }
    }
    out[i] = ranks_only ? k : mix(k + key_c);
  }
}

__global__ void k_exponential(uint64_t* out, uint64_t count, uint64_t start, uint64_t seed, double lam) {
  const uint64_t base = stream_base(seed, 0xE4);
  GRID_STRIDE(i, count) {
    const double u = unit(rand64(base, start + i));
    out[i] = (uint64_t)floor(-log1p(-u) / lam);
  }
}

struct Mix8 {
  double cw[8], mean[8], sigma[8];
  int k;
};

__global__ void k_gauss_mix(uint64_t* out, uint64_t count, uint64_t start, uint64_t seed, Mix8 m) {
  const uint64_t b0 = stream_base(seed, 0x6B), b1 = stream_base(seed, 0x6C), b2 = stream_base(seed, 0x6D);
  GRID_STRIDE(i, count) {
    const uint64_t idx = start + i;
    const double u0 = unit(rand64(b0, idx));
    int c = 0;
    while (c < m.k - 1 && u0 >= m.cw[c]) ++c;
    const double u1 = unit(rand64(b1, idx)), u2 = unit(rand64(b2, idx));
    const double z = sqrt(-2.0 * log1p(-u1)) * cospi(2.0 * u2);
    double x = m.mean[c] + m.sigma[c] * z;
    x = x < 0.0 ? 0.0 : (x > 18446744073709549568.0 ? 18446744073709549568.0 : x);
    out[i] = (uint64_t)floor(x);
  }
}

__global__ void k_rmat(uint32_t* src, uint32_t* dst, uint64_t count, uint64_t start, uint64_t seed, int scale,
                       double a, double b, double c) {
  GRID_STRIDE(i, count) {
    const uint64_t idx = start + i;
    uint32_t s = 0, d = 0;
    for (int l = 0; l < scale; ++l) {
      const double u = unit(rand64(stream_base(seed, 0x7000 + l), idx));
      const uint32_t row = u >= a + b;
      const uint32_t col = (u >= a && u < a + b) || (u >= a + b + c);
      s = (s << 1) | row;
      d = (d << 1) | col;
    }
    src[i] = s;
    dst[i] = d;
  }
}

unsigned grid_for(uint64_t count) {
  uint64_t g = (count + 255) / 256;
  return (unsigned)(g > 152 * 64 ? 152 * 64 : (g ? g : 1));
}

}  // namespace

extern "C" {

int synth_iota_u64(uint64_t* out, uint64_t count, uint64_t start, cudaStream_t st) {
  k_iota<<<grid_for(count), 256, 0, st>>>(out, count, start);
  return (int)cudaGetLastError();
}

int synth_iota_u32(uint32_t* out, uint64_t count, uint64_t start, cudaStream_t st) {
  k_iota32<<<grid_for(count), 256, 0, st>>>(out, count, start);
  return (int)cudaGetLastError();
}

int synth_uniform_mod(uint64_t* out, uint64_t count, uint64_t start, uint64_t seed, uint64_t mu, cudaStream_t st) {
  k_uniform_mod<<<grid_for(count), 256, 0, st>>>(out, count, start, seed, mu);
  return (int)cudaGetLastError();
}

int synth_uniform_exact(uint64_t* out, uint64_t count, uint64_t start, uint64_t n, uint64_t mu, uint64_t seed,
                        cudaStream_t st) {
  Feistel f;
  uint32_t bits = 2;
  while ((1ull << bits) < n) ++bits;
  if (bits % 2) ++bits;
  f.half = bits / 2;
  f.mask = (1ull << f.half) - 1;
  for (int r = 0; r < 4; ++r) f.rk[r] = stream_base(seed, 0xFE15 + r);
  k_uniform_exact<<<grid_for(count), 256, 0, st>>>(out, count, start, n, mu, f, stream_base(seed, 0x4B4559));
  return (int)cudaGetLastError();
}

int synth_zipf(uint64_t* out, uint64_t count, uint64_t start, uint64_t seed, double s, uint64_t N,
               double hx1, double hn, double sq, int ranks_only, cudaStream_t st) {
  ZipfP z{s, hx1, hn, sq, N};
  k_zipf<<<grid_for(count), 256, 0, st>>>(out, count, start, seed, z, stream_base(seed, 0x4B4559), ranks_only);
  return (int)cudaGetLastError();
}

int synth_exponential(uint64_t* out, uint64_t count, uint64_t start, uint64_t seed, double lam, cudaStream_t st) {
  k_exponential<<<grid_for(count), 256, 0, st>>>(out, count, start, seed, lam);
  return (int)cudaGetLastError();
}

int synth_gaussian_mixture(uint64_t* out, uint64_t count, uint64_t start, uint64_t seed, const double* cw,
                           const double* mean, const double* sigma, int k, cudaStream_t st) {
  Mix8 m;
  m.k = k > 8 ? 8 : k;
  for (int i = 0; i < m.k; ++i) {
    m.cw[i] = cw[i];
    m.mean[i] = mean[i];
    m.sigma[i] = sigma[i];
  }
  k_gauss_mix<<<grid_for(count), 256, 0, st>>>(out, count, start, seed, m);
  return (int)cudaGetLastError();
}

int synth_rmat(uint32_t* src, uint32_t* dst, uint64_t count, uint64_t start, uint64_t seed, int scale, double a,
               double b, double c, cudaStream_t st) {
  k_rmat<<<grid_for(count), 256, 0, st>>>(src, dst, count, start, seed, scale, a, b, c);
  return (int)cudaGetLastError();
}

}  // extern "C"
