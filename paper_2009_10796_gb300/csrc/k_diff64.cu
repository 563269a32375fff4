// FP64 instantiation of the differentiable forward and of its adjoint.
//
// The same computation as ddgi_diff_forward / ddgi_diff_backward (n frames
// of the update from a zero atlas with hysteresis 0, every probe tracing,
// then the query at fixed points), with everything that depends on the
// parameters (emitter radiance, object albedo) in double precision: hit
// shading (emitters, sun, the previous frame's probes at the hit), the
// normalised cosine / power-cosine averages with the gamma encoding of
// Sec. 4.2, the border copy of Sec. 7.1 and the 8-probe query of Sec. 2.2.
// Geometry is a constant of the parameters and keeps the FP32 traversal
// (closest hits, shadow rays; one ray per thread over the binary
// hierarchy), so central differences of this forward isolate the adjoint's
// own arithmetic: they are the FP64 check of the adjoint.
//
// Layouts: atlases [P][(n+2)^2][3] (irradiance) and [P][(m+2)^2][2]
// (distance moments) in double; ray records [P*R][4] (r, g, b, d).
#include "traverse.cuh"

namespace ddgi {

namespace {

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3(double x, double y, double z) { return D3{x, y, z}; }
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return d3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ D3 operator*(double s, D3 a) { return d3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double len(D3 a) { return sqrt(dot(a, a)); }
__device__ __forceinline__ D3 of(float3 a) { return d3(a.x, a.y, a.z); }
__device__ __forceinline__ D3 of(float4 a) { return d3(a.x, a.y, a.z); }

// Octahedral map (Cigolle et al. 2014), sign(0) = +1.
__device__ void oct64(D3 v, double& px, double& py) {
    const double l1 = fabs(v.x) + fabs(v.y) + fabs(v.z);
    px = v.x / l1;
    py = v.y / l1;
    if (v.z < 0.0) {
        const double qx = (1.0 - fabs(py)) * (px >= 0.0 ? 1.0 : -1.0);
        const double qy = (1.0 - fabs(px)) * (py >= 0.0 ? 1.0 : -1.0);
        px = qx;
        py = qy;
    }
}

// Direction of interior texel t of an n x n tile: the decoded centre.
__device__ D3 texel_dir64(int t, int n) {
    const int i = t % n, j = t / n;
    const double ux = 2.0 * (i + 0.5) / n - 1.0, uy = 2.0 * (j + 0.5) / n - 1.0;
    double x = ux, y = uy, z = 1.0 - fabs(ux) - fabs(uy);
    if (z < 0.0) {
        x = (1.0 - fabs(uy)) * (ux >= 0.0 ? 1.0 : -1.0);
        y = (1.0 - fabs(ux)) * (uy >= 0.0 ? 1.0 : -1.0);
    }
    const double l = sqrt(x * x + y * y + z * z);
    return d3(x / l, y / l, z / l);
}

// Bilinear footprint of an octahedral coordinate in a bordered tile of n
// interior texels: [-1, 1] spans texel positions [1, n + 1].
struct Fp64 {
    int x0, y0;
    double w[4];   // taps (x0, y0), (x0 + 1, y0), (x0, y0 + 1), (x0 + 1, y0 + 1)
};
__device__ Fp64 footprint64(double ux, double uy, int n) {
    const double sx = 1.0 + (ux + 1.0) * 0.5 * n - 0.5, sy = 1.0 + (uy + 1.0) * 0.5 * n - 0.5;
    Fp64 f;
    f.x0 = min(max((int)floor(sx), 0), n);
    f.y0 = min(max((int)floor(sy), 0), n);
    const double tx = sx - f.x0, ty = sy - f.y0;
    f.w[0] = (1.0 - tx) * (1.0 - ty);
    f.w[1] = tx * (1.0 - ty);
    f.w[2] = (1.0 - tx) * ty;
    f.w[3] = tx * ty;
    return f;
}
__device__ __forceinline__ int tap(const Fp64& f, int j, int N) { return (f.y0 + (j >> 1)) * N + f.x0 + (j & 1); }

// A volume of the differentiable path in double: grid, parameters, atlases.
struct View64 {
    D3 origin, spacing;
    int cx, cy, cz;
    double min_spacing, bias, gamma, t_max, cos_power;
    int ni, nd;
    const double* irr;    // [P][(ni+2)^2][3]
    const double* dist;   // [P][(nd+2)^2][2]
};

// The query's weights at x (normal n, towards w_o): the cage's probes, their
// weights w = trilinear x backface x max(Chebyshev, 1e-6) and the irradiance
// footprint of n (every probe of the differentiable volume is active).
struct Cage64 {
    int p[8];
    double w[8];
    Fp64 fn;
};
__device__ Cage64 cage64(const View64& v, D3 x, D3 n, D3 wo) {
    const double k = 0.75 * v.min_spacing * v.bias;
    const D3 xb = x + k * (0.2 * n + 0.8 * wo);
    const double g[3] = {(xb.x - v.origin.x) / v.spacing.x, (xb.y - v.origin.y) / v.spacing.y,
                         (xb.z - v.origin.z) / v.spacing.z};
    const int cnt[3] = {v.cx, v.cy, v.cz};
    int base[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        double b = floor(g[a]);
        b = fmin(fmax(b, 0.0), (double)(cnt[a] - 2));
        base[a] = (int)b;
        fr[a] = fmin(fmax(g[a] - b, 0.0), 1.0);
    }
    Cage64 c;
    double ux, uy;
    oct64(n, ux, uy);
    c.fn = footprint64(ux, uy, v.ni);
    const int M = v.nd + 2, tile_d = M * M;
    for (int q = 0; q < 8; ++q) {
        const int o[3] = {q & 1, (q >> 1) & 1, (q >> 2) & 1};
        const int i = base[0] + o[0], j = base[1] + o[1], kk = base[2] + o[2];
        const int p = i + v.cx * (j + v.cy * kk);
        const D3 xp = d3(v.origin.x + i * v.spacing.x, v.origin.y + j * v.spacing.y, v.origin.z + kk * v.spacing.z);
        double wt = 1.0;
        for (int a = 0; a < 3; ++a) wt *= o[a] ? fr[a] : 1.0 - fr[a];
        const D3 dp = xp - x;
        const double ldp = len(dp);
        const double cw = ldp > 0.0 ? dot(n, dp) / ldp : 1.0;
        const double hb = 0.5 * (1.0 + cw);
        const double wb = hb * hb + 0.2;
        const D3 pv = xb - xp;
        const double r = len(pv);
        double wc = 1.0;
        if (r > 0.0) {
            double vx, vy;
            oct64((1.0 / r) * pv, vx, vy);
            const Fp64 fd = footprint64(vx, vy, v.nd);
            double mu = 0.0, mu2 = 0.0;
            for (int jt = 0; jt < 4; ++jt) {
                const double* m = v.dist + ((int64_t)p * tile_d + tap(fd, jt, M)) * 2;
                mu += fd.w[jt] * m[0];
                mu2 += fd.w[jt] * m[1];
            }
            if (r > mu) {
                const double var = fmax(mu2 - mu * mu, 0.0);
                wc = var / (var + (r - mu) * (r - mu));
            }
        }
        c.p[q] = p;
        c.w[q] = wt * wb * fmax(wc, 1e-6);
    }
    return c;
}

// Bilinear irradiance sample b (gamma-encoded) of probe p at footprint f.
__device__ D3 irr_sample64(const View64& v, int p, const Fp64& f) {
    const int N = v.ni + 2;
    D3 b = d3(0.0, 0.0, 0.0);
    for (int j = 0; j < 4; ++j) {
        const double* e = v.irr + ((int64_t)p * N * N + tap(f, j, N)) * 3;
        b = b + f.w[j] * d3(e[0], e[1], e[2]);
    }
    return b;
}

__device__ __forceinline__ double decode_half(double b, double half_gamma) { return b > 0.0 ? pow(b, half_gamma) : 0.0; }

// Cosine-weighted mean radiance M = (sum w a / sum w)^2, a = b^(gamma/2).
__device__ D3 query_M64(const View64& v, D3 x, D3 n, D3 wo) {
    const Cage64 c = cage64(v, x, n, wo);
    const double hg = 0.5 * v.gamma;
    double sw = 0.0;
    D3 acc = d3(0.0, 0.0, 0.0);
    for (int q = 0; q < 8; ++q) {
        const D3 b = irr_sample64(v, c.p[q], c.fn);
        acc = acc + c.w[q] * d3(decode_half(b.x, hg), decode_half(b.y, hg), decode_half(b.z, hg));
        sw += c.w[q];
    }
    if (!(sw > 0.0)) return d3(0.0, 0.0, 0.0);
    const D3 A = (1.0 / sw) * acc;
    return d3(A.x * A.x, A.y * A.y, A.z * A.z);
}

// Reverse of query_M64: dM -> gradients of the irradiance texels (atomics).
__device__ void query_M64_adjoint(const View64& v, D3 x, D3 n, D3 wo, D3 dM, double* g_irr) {
    const Cage64 c = cage64(v, x, n, wo);
    const double hg = 0.5 * v.gamma;
    const int N = v.ni + 2;
    double sw = 0.0;
    D3 acc = d3(0.0, 0.0, 0.0), b8[8];
    for (int q = 0; q < 8; ++q) {
        b8[q] = irr_sample64(v, c.p[q], c.fn);
        acc = acc + c.w[q] * d3(decode_half(b8[q].x, hg), decode_half(b8[q].y, hg), decode_half(b8[q].z, hg));
        sw += c.w[q];
    }
    if (!(sw > 0.0)) return;
    const double A[3] = {acc.x / sw, acc.y / sw, acc.z / sw};
    const double dm[3] = {dM.x, dM.y, dM.z};
    for (int q = 0; q < 8; ++q) {
        const double bb[3] = {b8[q].x, b8[q].y, b8[q].z};
        for (int ch = 0; ch < 3; ++ch) {
            if (!(bb[ch] > 0.0)) continue;
            // dM/dA = 2A; dA/da_q = w_q / sw; da/db = (gamma/2) b^(gamma/2 - 1)
            const double d = dm[ch] * 2.0 * A[ch] * c.w[q] / sw * hg * pow(bb[ch], hg - 1.0);
            for (int j = 0; j < 4; ++j)
                atomicAdd(g_irr + ((int64_t)c.p[q] * N * N + tap(c.fn, j, N)) * 3 + ch, d * c.fn.w[j]);
        }
    }
}

// Closest hit of a probe ray in FP32 (the constant geometry) and its shading
// inputs in double.
struct Shade64 {
    int kind;        // 0 miss, 1 back face, 2 front face
    double t;
    D3 x, n;
    int obj, em;
    bool lit;        // front face facing the sun, shadow ray unblocked
    double cosl;
};
__device__ Shade64 trace64(const DevScene& s, const Lights& L, float3 of32, float3 df32) {
    Shade64 r{};
    const Hit h = traverse<false>(s, ray_pre(of32, df32));
    if (h.orig < 0) return r;
    const float4* T = s.tris + 3 * (int64_t)h.k;
    const float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
    const D3 e1 = of(p1) - of(p0), e2 = of(p2) - of(p0);
    const D3 ng = d3(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
    const D3 d = of(df32);
    r.t = h.t;
    if (dot(d, ng) > 0.0) {
        r.kind = 1;
        return r;
    }
    r.kind = 2;
    r.n = (1.0 / len(ng)) * ng;
    r.x = of(of32) + (double)h.t * d;
    const int2 at = __ldg(s.attr + h.orig);
    r.obj = at.x;
    r.em = at.y;
    const D3 tol = d3(-L.sun_dir.x, -L.sun_dir.y, -L.sun_dir.z);
    r.cosl = dot(r.n, tol);
    if (L.sun_on && r.cosl > 0.0) {
        const D3 so = r.x + (1e-4 * (1.0 + len(r.x))) * r.n;
        const Hit hs = traverse<true>(s, ray_pre(make_float3((float)so.x, (float)so.y, (float)so.z),
                                                 make_float3(-L.sun_dir.x, -L.sun_dir.y, -L.sun_dir.z)));
        r.lit = hs.orig < 0;
    }
    return r;
}

__device__ __forceinline__ float3 probe_pos_f32(const View64& v, int p) {
    const int i = p % v.cx, j = (p / v.cx) % v.cy, k = p / (v.cx * v.cy);
    return make_float3((float)(v.origin.x + i * v.spacing.x), (float)(v.origin.y + j * v.spacing.y),
                       (float)(v.origin.z + k * v.spacing.z));
}

// Thread per (probe, ray): the ray's record (r, g, b, d) in double.
__global__ void k_shade64(DevScene s, View64 prev, int with_prev, Lights L, const float4* __restrict__ dirs, int P,
                          int R, const double* __restrict__ albedo, const double* __restrict__ emit, double* rec) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)P * R;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx / R), i = (int)(idx - (int64_t)p * R);
        const float4 d4 = __ldg(dirs + i);
        const float3 o = probe_pos_f32(prev, p);
        const Shade64 h = trace64(s, L, o, make_float3(d4.x, d4.y, d4.z));
        const D3 d = of(d4);
        double out[4];
        if (h.kind == 0) {
            const double c = dot(d, of(L.sky_up));
            out[0] = L.sky_a.x + L.sky_b.x * c;
            out[1] = L.sky_a.y + L.sky_b.y * c;
            out[2] = L.sky_a.z + L.sky_b.z * c;
            out[3] = prev.t_max;
        } else if (h.kind == 1) {
            out[0] = out[1] = out[2] = 0.0;
            out[3] = fmin(0.2 * h.t, prev.t_max);
        } else {
            const double* rho = albedo + 3 * (int64_t)h.obj;
            const double kk = h.lit ? h.cosl / 3.14159265358979323846 : 0.0;
            const D3 direct = kk * of(L.sun_irr);
            const D3 M = with_prev ? query_M64(prev, h.x, h.n, d3(-d.x, -d.y, -d.z)) : d3(0.0, 0.0, 0.0);
            const D3 Le = h.em >= 0 ? d3(emit[3 * h.em], emit[3 * h.em + 1], emit[3 * h.em + 2]) : d3(0.0, 0.0, 0.0);
            out[0] = Le.x + rho[0] * (direct.x + M.x);
            out[1] = Le.y + rho[1] * (direct.y + M.y);
            out[2] = Le.z + rho[2] * (direct.z + M.z);
            out[3] = fmin((double)h.t, prev.t_max);
        }
        for (int k = 0; k < 4; ++k) rec[4 * idx + k] = out[k];
    }
}

// Normalised weight sums of texel t over the rays (irradiance: cosine;
// distance: cosine^p).
__device__ __forceinline__ double weight64(D3 nt, const float4* dirs, int i, bool is_irr, double p) {
    const double c = fmax(0.0, dot(nt, of(__ldg(dirs + i))));
    return is_irr ? c : pow(c, p);
}

// Block per probe, thread per texel: the new tile (hysteresis 0: e = m^(1/gamma)
// for irradiance, the moments for distance) and its border copies.
__global__ void k_blend64(View64 v, const float4* __restrict__ dirs, int R, const double* __restrict__ rec,
                          double* irr_out, double* dist_out) {
    const int p = blockIdx.x;
    const int ti = v.ni * v.ni, td = v.nd * v.nd, N = v.ni + 2, M = v.nd + 2;
    const double* rp = rec + (int64_t)p * R * 4;
    for (int t = threadIdx.x; t < ti + td; t += blockDim.x) {
        const bool is_irr = t < ti;
        const int u = is_irr ? t : t - ti, n = is_irr ? v.ni : v.nd;
        const D3 nt = texel_dir64(u, n);
        double sw = 0.0, a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int i = 0; i < R; ++i) {
            const double w = weight64(nt, dirs, i, is_irr, v.cos_power);
            sw += w;
            if (is_irr) {
                a0 += w * rp[4 * i];
                a1 += w * rp[4 * i + 1];
                a2 += w * rp[4 * i + 2];
            } else {
                const double dd = rp[4 * i + 3];
                a0 += w * dd;
                a1 += w * dd * dd;
            }
        }
        if (!(sw > 0.0)) continue;   // unreached texel: keeps its value (zero atlas)
        const int x = 1 + u % n, y = 1 + u / n;
        double e[3];
        if (is_irr) {
            e[0] = pow(a0 / sw, 1.0 / v.gamma);
            e[1] = pow(a1 / sw, 1.0 / v.gamma);
            e[2] = pow(a2 / sw, 1.0 / v.gamma);
        } else {
            e[0] = a0 / sw;
            e[1] = a1 / sw;
        }
        const int C = is_irr ? 3 : 2, W = is_irr ? N : M;
        double* tile = (is_irr ? irr_out + (int64_t)p * N * N * 3 : dist_out + (int64_t)p * M * M * 2);
        auto put = [&](int bx, int by) {
            for (int c = 0; c < C; ++c) tile[(by * W + bx) * C + c] = e[c];
        };
        put(x, y);
        if (x == 1) put(0, n + 1 - y);
        if (x == n) put(n + 1, n + 1 - y);
        if (y == 1) put(n + 1 - x, 0);
        if (y == n) put(n + 1 - x, n + 1);
        if (x == n && y == n) put(0, 0);
        if (x == 1 && y == n) put(n + 1, 0);
        if (x == n && y == 1) put(0, n + 1);
        if (x == 1 && y == 1) put(n + 1, n + 1);
    }
}

__device__ __forceinline__ D3 view_dir64(float3 cam, D3 x, D3 n) {
    D3 wo = of(cam) - x;
    const double l = len(wo);
    return l < 1e-6 ? n : (1.0 / l) * wo;
}

// E = pi M at n points (a zero normal gives 0).
__global__ void k_query64(View64 v, const float* __restrict__ pos, const float* __restrict__ nrm, int64_t n,
                          float3 cam, double* out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const D3 x = d3(pos[3 * q], pos[3 * q + 1], pos[3 * q + 2]);
        const D3 nn = d3(nrm[3 * q], nrm[3 * q + 1], nrm[3 * q + 2]);
        D3 E = d3(0.0, 0.0, 0.0);
        if (nn.x != 0.0 || nn.y != 0.0 || nn.z != 0.0)
            E = 3.14159265358979323846 * query_M64(v, x, nn, view_dir64(cam, x, nn));
        out[3 * q] = E.x;
        out[3 * q + 1] = E.y;
        out[3 * q + 2] = E.z;
    }
}

__global__ void k_query_adjoint64(View64 v, const float* __restrict__ pos, const float* __restrict__ nrm, int64_t n,
                                  float3 cam, const double* __restrict__ dE, double* g_irr) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const D3 x = d3(pos[3 * q], pos[3 * q + 1], pos[3 * q + 2]);
        const D3 nn = d3(nrm[3 * q], nrm[3 * q + 1], nrm[3 * q + 2]);
        if (nn.x == 0.0 && nn.y == 0.0 && nn.z == 0.0) continue;
        const double pi = 3.14159265358979323846;
        query_M64_adjoint(v, x, nn, view_dir64(cam, x, nn), d3(pi * dE[3 * q], pi * dE[3 * q + 1], pi * dE[3 * q + 2]),
                          g_irr);
    }
}

// Block per probe: border gradients folded into the interior texels they copy.
__global__ void k_border_fold64(double* g_irr, int n) {
    const int N = n + 2;
    double* t = g_irr + (int64_t)blockIdx.x * N * N * 3;
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
        const int x = 1 + q % n, y = 1 + q / n;
        double add[3] = {0.0, 0.0, 0.0};
        auto gather = [&](int bx, int by) {
            for (int c = 0; c < 3; ++c) add[c] += t[(by * N + bx) * 3 + c];
        };
        if (x == 1) gather(0, n + 1 - y);
        if (x == n) gather(n + 1, n + 1 - y);
        if (y == 1) gather(n + 1 - x, 0);
        if (y == n) gather(n + 1 - x, n + 1);
        if (x == n && y == n) gather(0, 0);
        if (x == 1 && y == n) gather(n + 1, 0);
        if (x == n && y == 1) gather(0, n + 1);
        if (x == 1 && y == 1) gather(n + 1, n + 1);
        for (int c = 0; c < 3; ++c) t[(y * N + x) * 3 + c] += add[c];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
        const int x = q % N, y = q / N;
        if (x == 0 || y == 0 || x == N - 1 || y == N - 1)
            for (int c = 0; c < 3; ++c) t[q * 3 + c] = 0.0;
    }
}

// Thread per irradiance texel: s_t = sum_i max(0, n_t . w_i).
__global__ void k_rowsum64(int ni, const float4* __restrict__ dirs, int R, double* s) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ni * ni) return;
    const D3 nt = texel_dir64(t, ni);
    double a = 0.0;
    for (int i = 0; i < R; ++i) a += weight64(nt, dirs, i, true, 1.0);
    s[t] = a;
}

// Thread per (probe, ray): dL_i = sum_t (w_ti / s_t) de/dm g_t, e = m^(1/gamma)
// the texel value this frame wrote (de/dm = (1/gamma) e^(1 - gamma)).
__global__ void k_blend_adjoint64(View64 v_after, const float4* __restrict__ dirs, int P, int R,
                                  const double* __restrict__ sw_irr, const double* __restrict__ g_irr, double* gL) {
    const int ni = v_after.ni, N = ni + 2, ti = ni * ni;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)P * R;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx / R), i = (int)(idx - (int64_t)p * R);
        double a[3] = {0.0, 0.0, 0.0};
        for (int t = 0; t < ti; ++t) {
            const D3 nt = texel_dir64(t, ni);
            const double w = weight64(nt, dirs, i, true, 1.0);
            const double sw = sw_irr[t];
            if (w == 0.0 || !(sw > 0.0)) continue;
            const int x = 1 + t % ni, y = 1 + t / ni;
            const double* gg = g_irr + ((int64_t)p * N * N + y * N + x) * 3;
            const double* e = v_after.irr + ((int64_t)p * N * N + y * N + x) * 3;
            for (int c = 0; c < 3; ++c) {
                const double d = e[c] > 0.0 ? pow(e[c], 1.0 - v_after.gamma) / v_after.gamma
                                            : (v_after.gamma == 1.0 ? 1.0 : 0.0);
                a[c] += w / sw * d * gg[c];
            }
        }
        for (int c = 0; c < 3; ++c) gL[4 * idx + c] = a[c];
        gL[4 * idx + 3] = 0.0;
    }
}

// Thread per (probe, ray) of a frame, traced again: the emitter term on
// front hits, the albedo term (direct + previous-frame query), and rho dL
// into the previous frame's query adjoint.
__global__ void k_shade_adjoint64(DevScene s, View64 v_before, int with_prev, Lights L,
                                  const float4* __restrict__ dirs, int P, int R, const double* __restrict__ albedo,
                                  const double* __restrict__ gL, double* d_emit, double* d_albedo, double* g_prev) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)P * R;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const D3 g = d3(gL[4 * idx], gL[4 * idx + 1], gL[4 * idx + 2]);
        if (g.x == 0.0 && g.y == 0.0 && g.z == 0.0) continue;
        const int p = (int)(idx / R), i = (int)(idx - (int64_t)p * R);
        const float4 d4 = __ldg(dirs + i);
        const Shade64 h = trace64(s, L, probe_pos_f32(v_before, p), make_float3(d4.x, d4.y, d4.z));
        if (h.kind != 2) continue;
        if (h.em >= 0) {
            atomicAdd(d_emit + 3 * h.em, g.x);
            atomicAdd(d_emit + 3 * h.em + 1, g.y);
            atomicAdd(d_emit + 3 * h.em + 2, g.z);
        }
        const double kk = h.lit ? h.cosl / 3.14159265358979323846 : 0.0;
        const D3 direct = kk * of(L.sun_irr);
        const D3 wo = d3(-d4.x, -d4.y, -d4.z);
        const D3 M = with_prev ? query_M64(v_before, h.x, h.n, wo) : d3(0.0, 0.0, 0.0);
        atomicAdd(d_albedo + 3 * h.obj, g.x * (direct.x + M.x));
        atomicAdd(d_albedo + 3 * h.obj + 1, g.y * (direct.y + M.y));
        atomicAdd(d_albedo + 3 * h.obj + 2, g.z * (direct.z + M.z));
        if (with_prev) {
            const double* rho = albedo + 3 * (int64_t)h.obj;
            query_M64_adjoint(v_before, h.x, h.n, wo, d3(g.x * rho[0], g.y * rho[1], g.z * rho[2]), g_prev);
        }
    }
}

int grid64(int64_t n, int block) {
    const int64_t b = (n + block - 1) / block;
    return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

View64 view64(const Diff64Volume& dv, const double* irr, const double* dist) {
    View64 v;
    v.origin = D3{dv.origin[0], dv.origin[1], dv.origin[2]};
    v.spacing = D3{dv.spacing[0], dv.spacing[1], dv.spacing[2]};
    v.cx = dv.counts[0];
    v.cy = dv.counts[1];
    v.cz = dv.counts[2];
    v.min_spacing = fmin(dv.spacing[0], fmin(dv.spacing[1], dv.spacing[2]));
    v.bias = dv.bias;
    v.gamma = dv.gamma;
    v.t_max = dv.t_max;
    v.cos_power = dv.cos_power;
    v.ni = dv.irr_n;
    v.nd = dv.dist_n;
    v.irr = irr;
    v.dist = dist;
    return v;
}

}  // namespace

cudaError_t launch_diff64_frame(const Diff64Volume& dv, const DevScene& s, const Lights& L, const float4* dirs,
                                const double* albedo, const double* emit, const double* irr_prev,
                                const double* dist_prev, int with_prev, double* rec, double* irr_out,
                                double* dist_out, cudaStream_t st) {
    const int P = dv.counts[0] * dv.counts[1] * dv.counts[2];
    const int64_t n = (int64_t)P * dv.R;
    k_shade64<<<grid64(n, 128), 128, 0, st>>>(s, view64(dv, irr_prev, dist_prev), with_prev, L, dirs, P, dv.R, albedo,
                                              emit, rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_blend64<<<P, 256, 0, st>>>(view64(dv, nullptr, nullptr), dirs, dv.R, rec, irr_out, dist_out);
    return cudaGetLastError();
}

cudaError_t launch_diff64_query(const Diff64Volume& dv, const double* irr, const double* dist, const float* pos,
                                const float* nrm, int64_t n, float3 cam, double* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_query64<<<grid64(n, 128), 128, 0, st>>>(view64(dv, irr, dist), pos, nrm, n, cam, out);
    return cudaGetLastError();
}

cudaError_t launch_diff64_query_adjoint(const Diff64Volume& dv, const double* irr, const double* dist,
                                        const float* pos, const float* nrm, int64_t n, float3 cam, const double* dE,
                                        double* g_irr, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_query_adjoint64<<<grid64(n, 128), 128, 0, st>>>(view64(dv, irr, dist), pos, nrm, n, cam, dE, g_irr);
    return cudaGetLastError();
}

cudaError_t launch_diff64_frame_adjoint(const Diff64Volume& dv, const DevScene& s, const Lights& L,
                                        const float4* dirs, const double* albedo, const double* irr_before,
                                        const double* dist_before, const double* irr_after, int with_prev,
                                        double* sw_irr, double* g_irr, double* gL, double* d_emit, double* d_albedo,
                                        double* g_prev, cudaStream_t st) {
    const int P = dv.counts[0] * dv.counts[1] * dv.counts[2];
    const int64_t n = (int64_t)P * dv.R;
    k_border_fold64<<<P, 64, 0, st>>>(g_irr, dv.irr_n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_rowsum64<<<(dv.irr_n * dv.irr_n + 127) / 128, 128, 0, st>>>(dv.irr_n, dirs, dv.R, sw_irr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_blend_adjoint64<<<grid64(n, 128), 128, 0, st>>>(view64(dv, irr_after, nullptr), dirs, P, dv.R, sw_irr, g_irr,
                                                      gL);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_shade_adjoint64<<<grid64(n, 128), 128, 0, st>>>(s, view64(dv, irr_before, dist_before), with_prev, L, dirs, P,
                                                      dv.R, albedo, gL, d_emit, d_albedo, g_prev);
    return cudaGetLastError();
}

}  // namespace ddgi
