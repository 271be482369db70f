// pst.cu -- particle swarm template pre-sampling (Sec. 4, "PST pre-sampling").
//
// The PST is a fixed set of points in the closed unit 6D ball (Sec. 3.3: c_0 = 0,
// r_0 = 1); row 0 is the origin so that particle 0 always sits on the PST centre.
// Method 0 draws every particle independently by rejection from the cube with a
// counter-based generator (Philox4x32-10, Salmon et al., SC 2011), one thread per
// particle; method 1 is Poisson-disk sampling after Bridson (SIGGRAPH 2007
// sketch), inherently sequential and therefore run on the host.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace rf {

// Philox4x32 with 10 rounds: per round two 32x32 -> 64-bit products of the
// counter words 0 and 2 with 0xD2511F53 and 0xCD9E8D57, the high halves xor-ed
// with the other two words and the key; the key is bumped by the Weyl
// increments 0x9E3779B9 and 0xBB67AE85 between rounds.
struct Philox {
    __host__ __device__ static void round(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0,
                                          uint32_t k1)
    {
        const uint64_t a = (uint64_t)c0 * 0xD2511F53ull;
        const uint64_t b = (uint64_t)c2 * 0xCD9E8D57ull;
        const uint32_t n0 = (uint32_t)(b >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)b;
        c3 = (uint32_t)a;
        c0 = n0;
        c2 = n2;
    }
    __host__ __device__ static void eval(const uint32_t in[4], uint32_t k0, uint32_t k1, uint32_t out[4])
    {
        uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            round(c0, c1, c2, c3, k0, k1);
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        out[0] = c0;
        out[1] = c1;
        out[2] = c2;
        out[3] = c3;
    }
};

// Uniform sampler.  Particle i >= 1, attempt a: words of Philox((i, a, 0, 0)) and
// Philox((i, a, 1, 0)) under key = seed; coordinate d is (2 m_d + 1 - 2^24) / 2^24
// with m_d the top 24 bits of word d, which float32 holds exactly; accepted iff
// sum_d (2 m_d + 1 - 2^24)^2 <= 2^48, decided in exact 64-bit integers.
__global__ void pst_uniform_kernel(int n, uint32_t k0, uint32_t k1, float *out, int *fail)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    if (i == 0) {
        for (int d = 0; d < 6; ++d)
            out[(size_t)d * n] = 0.f;
        return;
    }
    for (uint32_t a = 0; a < 100000u; ++a) {
        uint32_t w[8];
        const uint32_t c0[4] = {(uint32_t)i, a, 0u, 0u}, c1[4] = {(uint32_t)i, a, 1u, 0u};
        Philox::eval(c0, k0, k1, w);
        Philox::eval(c1, k0, k1, w + 4);
        long long v[6], s2 = 0;
        for (int d = 0; d < 6; ++d) {
            v[d] = 2ll * (long long)(w[d] >> 8) + 1ll - (1ll << 24);
            s2 += v[d] * v[d];
        }
        if (s2 <= (1ll << 48)) {
            for (int d = 0; d < 6; ++d)
                out[(size_t)d * n + i] = (float)v[d] * (1.0f / 16777216.0f);
            return;
        }
    }
    atomicExch(fail, 1);
    for (int d = 0; d < 6; ++d)
        out[(size_t)d * n + i] = 0.f;
}

// ------------------------------------------------------------------ Poisson disk (host)
// Bridson's algorithm in the unit 6D ball: a background grid with cell side r
// (so any neighbour closer than r lies in the 3^6 surrounding cells), an active
// list seeded with the origin, and up to 30 candidates per active sample drawn
// uniformly in the annulus [r, 2r] by rejection from the cube.  The radius is
// chosen by bisection so that the maximal sample holds at least n points; n - 1
// of them (plus the origin) are then kept by a Philox-driven partial shuffle.
namespace {

struct HostRng {
    uint32_t k0, k1, stream, ctr = 0, buf[4], pos = 4;
    uint32_t next()
    {
        if (pos == 4) {
            const uint32_t c[4] = {ctr++, stream, 0x5eed5eedu, 0u};
            Philox::eval(c, k0, k1, buf);
            pos = 0;
        }
        return buf[pos++];
    }
    double uniform() { return (next() >> 8) * (1.0 / 16777216.0); }  // [0, 1)
};

struct Grid {
    int cells;        // per axis
    double side, lo;  // cell side and lower bound (-1)
    std::vector<int> head;
    std::vector<int> next;
    int coord(double x) const
    {
        int c = (int)floor((x - lo) / side);
        return std::min(std::max(c, 0), cells - 1);
    }
    size_t key(const int c[6]) const
    {
        size_t k = 0;
        for (int d = 5; d >= 0; --d)
            k = k * cells + c[d];
        return k;
    }
};

int bridson(double r, uint32_t k0, uint32_t k1, int cap, std::vector<double> &pts)
{
    Grid g;
    g.side = r;
    g.lo = -1.0;
    g.cells = (int)ceil(2.0 / r);
    double total = pow((double)g.cells, 6.0);
    if (total > 6.0e7)
        return -1;
    g.head.assign((size_t)total, -1);
    g.next.clear();
    pts.clear();
    HostRng rng{k0, k1, (uint32_t)(r * 1e6)};
    auto insert = [&](const double *p) {
        int c[6];
        for (int d = 0; d < 6; ++d)
            c[d] = g.coord(p[d]);
        size_t k = g.key(c);
        int id = (int)(pts.size() / 6);
        pts.insert(pts.end(), p, p + 6);
        g.next.push_back(g.head[k]);
        g.head[k] = id;
        return id;
    };
    auto far_enough = [&](const double *p) {
        int c[6];
        for (int d = 0; d < 6; ++d)
            c[d] = g.coord(p[d]);
        int o[6];
        for (int idx = 0; idx < 729; ++idx) {
            int t = idx;
            bool ok = true;
            for (int d = 0; d < 6; ++d) {
                o[d] = c[d] + (t % 3) - 1;
                t /= 3;
                if (o[d] < 0 || o[d] >= g.cells)
                    ok = false;
            }
            if (!ok)
                continue;
            for (int j = g.head[g.key(o)]; j >= 0; j = g.next[j]) {
                double s = 0;
                for (int d = 0; d < 6; ++d) {
                    double e = pts[6 * (size_t)j + d] - p[d];
                    s += e * e;
                }
                if (s < r * r)
                    return false;
            }
        }
        return true;
    };
    const double origin[6] = {0, 0, 0, 0, 0, 0};
    std::vector<int> active{insert(origin)};
    while (!active.empty() && (int)(pts.size() / 6) < cap) {
        size_t ai = rng.next() % active.size();
        const int a = active[ai];
        bool placed = false;
        for (int tries = 0; tries < 30 && !placed; ++tries) {
            double c[6];
            for (int rej = 0; rej < 10000; ++rej) {
                double s = 0;
                for (int d = 0; d < 6; ++d) {
                    c[d] = (rng.uniform() * 2.0 - 1.0) * 2.0 * r;
                    s += c[d] * c[d];
                }
                if (s >= r * r && s <= 4.0 * r * r)
                    break;
            }
            double p[6], s = 0;
            for (int d = 0; d < 6; ++d) {
                p[d] = pts[6 * (size_t)a + d] + c[d];
                s += p[d] * p[d];
            }
            if (s <= 1.0 && far_enough(p)) {
                active.push_back(insert(p));
                placed = true;
            }
        }
        if (!placed) {
            active[ai] = active.back();
            active.pop_back();
        }
    }
    return (int)(pts.size() / 6);
}

}  // namespace

rf_status pst_poisson_host(int n, uint64_t seed, std::vector<float> &out, double *radius)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    std::vector<double> pts;
    double lo = 0.02, hi = 1.0, best_r = -1;
    std::vector<double> best;
    const int cap = 16 * n + 64;  // a capped run would be a blob around the origin: never kept
    for (int it = 0; it < 16; ++it) {
        double r = 0.5 * (lo + hi);
        int got = bridson(r, k0, k1, cap, pts);
        if (got < 0 || got >= cap) {
            lo = r;  // grid too fine or far too many points: the radius must grow
        } else if (got >= n) {
            best_r = r;
            best = pts;
            lo = r;
        } else {
            hi = r;
        }
        if (hi - lo < 1e-3 * hi && best_r > 0)
            break;
    }
    if (best_r < 0) {
        set_error("pst_create: Poisson-disk sampling did not reach %d points", n);
        return RF_ERR_ARG;
    }
    int m = (int)(best.size() / 6);
    std::vector<int> idx(m);
    for (int i = 0; i < m; ++i)
        idx[i] = i;
    HostRng rng{k0, k1, 0xabcdu};
    for (int i = 1; i < n; ++i) {  // keep idx[0] = origin
        int j = i + (int)(rng.next() % (uint32_t)(m - i));
        std::swap(idx[i], idx[j]);
    }
    out.assign((size_t)6 * n, 0.f);
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 6; ++d)
            out[(size_t)d * n + i] = (float)best[6 * (size_t)idx[i] + d];
    if (radius)
        *radius = best_r;
    return RF_OK;
}

}  // namespace rf

using namespace rf;

extern "C" rf_status pst_create(int n, uint64_t seed, int method, float *out_dev, void *stream)
{
    RF_CHECK_ARG(out_dev != nullptr, "null output");
    RF_CHECK_ARG(n >= 1, "n must be >= 1");
    RF_CHECK_ARG(method == 0 || method == 1, "method must be 0 (uniform) or 1 (Poisson disk)");
    cudaStream_t s = (cudaStream_t)stream;
    if (method == 0) {
        int *fail = nullptr;
        RF_CUDA(cudaMallocAsync(&fail, sizeof(int), s));
        RF_CUDA(cudaMemsetAsync(fail, 0, sizeof(int), s));
        pst_uniform_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, (uint32_t)seed, (uint32_t)(seed >> 32), out_dev, fail);
        RF_CUDA(cudaGetLastError());
        int h = 0;
        RF_CUDA(cudaMemcpyAsync(&h, fail, sizeof(int), cudaMemcpyDeviceToHost, s));
        RF_CUDA(cudaFreeAsync(fail, s));
        RF_CUDA(cudaStreamSynchronize(s));
        if (h) {
            set_error("pst_create: rejection sampling exhausted its attempts");
            return RF_ERR_ARG;
        }
        return RF_OK;
    }
    std::vector<float> host;
    rf_status st = pst_poisson_host(n, seed, host, nullptr);
    if (st != RF_OK)
        return st;
    RF_CUDA(cudaMemcpyAsync(out_dev, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    RF_CUDA(cudaStreamSynchronize(s));
    return RF_OK;
}
