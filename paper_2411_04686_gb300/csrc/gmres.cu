// gmres.cu -- stepped mixed-precision restarted GMRES(m) (Alg. 3, Sec. III-D)
// on the device: FP64 Arnoldi by classical Gram-Schmidt with one conditional
// re-orthogonalisation pass (the DGKS test ||w_after|| < 0.7 ||w_before||),
// Givens rotations and the least-squares residual estimate in a one-warp
// kernel, the update x += V y as one fused pass.
//
// The Krylov basis is kept unnormalised: V_j holds a vector and scale_j its
// inverse norm, so the normalisation folds into the dot products and updates
// instead of costing a pass over memory.  The level k changes only between
// cycles (changing A inside a cycle would break A V = V H); the host reads a
// few scalars once per cycle to take those decisions.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "pool.cuh"
#include "solver_internal.cuh"

namespace gse {

constexpr int GM_MAX_RESTART = 64;
constexpr int GM_RING_MAX = 4096;

struct GmState {
    int stop, i_done, j, need_reorth, hlen, hpos, lucky, pad;
    double nb, tol, res, wb2, wn, rsd, reldec, ndec;
    double scale[GM_MAX_RESTART + 1];
    double hcol[GM_MAX_RESTART + 1];
    double corr[GM_MAX_RESTART + 1];
    double R[(GM_MAX_RESTART + 1) * GM_MAX_RESTART];  // column i at R[i*(m+1) ...]
    double cs[GM_MAX_RESTART], sn[GM_MAX_RESTART];
    double g[GM_MAX_RESTART + 1], y[GM_MAX_RESTART];
};

__device__ __forceinline__ double gm_block_sum(double v, double* red) { return block_sum(v, red); }

// Deterministic grid sum of nvals values per thread; the last block gets the
// totals in sh_tot[0..nvals) (every thread) and returns true.
__device__ bool gm_grid_sums(const double* vals, int nvals, double* partial, unsigned* counter,
                             double* red, double* sh_tot) {
    __shared__ bool last;
    for (int j = 0; j < nvals; j++) {
        const double s = block_sum(vals[j], red);
        if (threadIdx.x == 0) partial[(size_t)j * gridDim.x + blockIdx.x] = s;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int j = 0; j < nvals; j++) {
        double a = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) a += __ldcg(partial + (size_t)j * gridDim.x + b);
        a = block_sum(a, red);
        if (threadIdx.x == 0) sh_tot[j] = a;
    }
    if (threadIdx.x == 0) *counter = 0;
    __syncthreads();
    return true;
}

// beta = ||v0||; starts a cycle.
__global__ void k_gm_start(GmState* st, const double* __restrict__ v0, int64_t n, double* partial,
                           unsigned* counter) {
    __shared__ double red[32];
    __shared__ double tot[1];
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        acc = fma(v0[t], v0[t], acc);
    if (!gm_grid_sums(&acc, 1, partial, counter, red, tot)) return;
    if (threadIdx.x == 0) {
        const double beta = sqrt(tot[0]);
        st->scale[0] = beta > 0.0 ? 1.0 / beta : 0.0;
        st->g[0] = beta;
        st->res = beta / st->nb;
        st->i_done = 0;
        st->lucky = 0;
        st->need_reorth = 0;
        st->stop = (!(st->res >= st->tol)) || beta == 0.0 ? 1 : 0;
        st->wn = beta;
    }
}

// ||v||^2 into st->wb2 (used for true residuals).
__global__ void k_gm_norm(GmState* st, const double* __restrict__ v, int64_t n, double* partial,
                          unsigned* counter) {
    __shared__ double red[32];
    __shared__ double tot[1];
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        acc = fma(v[t], v[t], acc);
    if (!gm_grid_sums(&acc, 1, partial, counter, red, tot)) return;
    if (threadIdx.x == 0) st->wb2 = tot[0];
}

// Dots of w = V[i+1] with V[0..i].  pass 0: w is A V_i unscaled; h_j =
// scale_i scale_j (w_raw . V_j) and ||w||^2 before orthogonalisation.
// pass 1 (re-orthogonalisation, only if flagged): c_j = scale_j (w . V_j).
// The i + 2 sums are taken 8 at a time in registers; block partials go to
// shared memory, then one grid-level reduction for all of them.
// Warp sums of 8 values per lane with 9 FP64 additions per lane (instead of 8
// separate 5-step reductions, 40 additions): at each of the first three
// exchanges a lane keeps half of its values and adds the partner's copy of
// them, then the last value is summed over the 4-lane group.  Afterwards lane
// L holds the full sum of value 4*bit4(L) + 2*bit3(L) + bit2(L).
__device__ __forceinline__ double warp_sum8(const double* a, int lane) {
    const unsigned FULL = 0xFFFFFFFFu;
    double b[4], c[2];
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const double send = h16 ? a[u] : a[u + 4];
        b[u] = (h16 ? a[u + 4] : a[u]) + __shfl_xor_sync(FULL, send, 16);
    }
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const double send = h8 ? b[u] : b[u + 2];
        c[u] = (h8 ? b[u + 2] : b[u]) + __shfl_xor_sync(FULL, send, 8);
    }
    double d = (h4 ? c[1] : c[0]) + __shfl_xor_sync(FULL, h4 ? c[0] : c[1], 4);
    d += __shfl_xor_sync(FULL, d, 2);
    d += __shfl_xor_sync(FULL, d, 1);
    return d;
}

// h_j = v_j . w for j <= i and |w|^2 (CGS step; pass 1 is the DGKS correction),
// 8 dot products per sweep over w.
__global__ void __launch_bounds__(256, 4) k_gm_dots(GmState* st, const double* __restrict__ V, int64_t n, int i,
                                                  int pass, double* partial, unsigned* counter) {
    __shared__ double bpart[GM_MAX_RESTART + 2];
    __shared__ double wsum[8][8];
    __shared__ bool last;
    if (st->stop || (pass == 1 && !st->need_reorth)) return;
    const double* w = V + (size_t)(i + 1) * n;
    const int nv = i + 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int jb = 0; jb < nv; jb += 8) {
        double a[8];
#pragma unroll
        for (int u = 0; u < 8; u++) a[u] = 0.0;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        // two elements per step, all their loads in flight together; each sum
        // still takes its terms in order of t
        for (; t + stride < n; t += 2 * stride) {
            const double w0 = w[t], w1 = w[t + stride];
            double v0[8], v1[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int j = jb + u;
                v0[u] = j <= i ? V[(size_t)j * n + t] : w0;
                v1[u] = j <= i ? V[(size_t)j * n + t + stride] : w1;
            }
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (jb + u < nv) a[u] = fma(w1, v1[u], fma(w0, v0[u], a[u]));
        }
        for (; t < n; t += stride) {
            const double wt = w[t];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int j = jb + u;
                if (j < nv) a[u] = fma(wt, j <= i ? V[(size_t)j * n + t] : wt, a[u]);
            }
        }
        const double d = warp_sum8(a, lane);
        if ((lane & 3) == 0) wsum[warp][((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] = d;
        __syncthreads();
        if (threadIdx.x < 8) {
            double sum = 0.0;
            for (int wi = 0; wi < (int)(blockDim.x >> 5); wi++) sum += wsum[wi][threadIdx.x];
            if (jb + (int)threadIdx.x < nv) bpart[jb + threadIdx.x] = sum;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int j = 0; j < nv; j++) partial[(size_t)j * gridDim.x + blockIdx.x] = bpart[j];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the columns' totals in parallel: one warp per column sums a lane-strided
    // slice of its per-block partials and reduces by shuffles (no block-wide
    // barrier per column in this serial tail)
    for (int j = warp; j < nv; j += (int)(blockDim.x >> 5)) {
        double a = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) a += __ldcg(partial + (size_t)j * gridDim.x + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        if (lane == 0) bpart[j] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *counter = 0;
        if (pass == 0) {
            const double si = st->scale[i];
            for (int j = 0; j <= i; j++) st->hcol[j] = si * st->scale[j] * bpart[j];
            st->wb2 = si * si * bpart[i + 1];
        } else {
            for (int j = 0; j <= i; j++) st->corr[j] = st->scale[j] * bpart[j];
        }
    }
}
__global__ void __launch_bounds__(256, 4) k_gm_axpy(GmState* st, double* __restrict__ V, int64_t n, int i, int pass,
                                                  double* partial, unsigned* counter) {
    __shared__ double red[32];
    __shared__ double tot[1];
    __shared__ double coef[GM_MAX_RESTART + 1];
    if (st->stop || (pass == 1 && !st->need_reorth)) return;
    for (int j = threadIdx.x; j <= i; j += blockDim.x)
        coef[j] = (pass == 0 ? st->hcol[j] : st->corr[j]) * st->scale[j];
    const double si = pass == 0 ? st->scale[i] : 1.0;
    __syncthreads();
    double* w = V + (size_t)(i + 1) * n;
    double acc = 0.0;
    // four elements per thread, so each basis vector contributes four
    // independent loads and FMAs (the chain over j is sequential per element)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t0 < n; t0 += 4 * stride) {
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] = t0 + q * stride < n ? si * w[t0 + q * stride] : 0.0;
        // two basis vectors' loads in flight per step (the FMA chain over j
        // keeps its order)
        int j = 0;
        for (; j + 1 <= i; j += 2) {
            const double* vj = V + (size_t)j * n;
            const double* vk = vj + n;
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const bool in = t0 + q * stride < n;
                a[q] = in ? vj[t0 + q * stride] : 0.0;
                b[q] = in ? vk[t0 + q * stride] : 0.0;
            }
            const double c = -coef[j], d = -coef[j + 1];
#pragma unroll
            for (int q = 0; q < 4; q++) v[q] = fma(d, b[q], fma(c, a[q], v[q]));
        }
        for (; j <= i; j++) {
            const double c = -coef[j];
            const double* vj = V + (size_t)j * n;
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (t0 + q * stride < n) v[q] = fma(c, vj[t0 + q * stride], v[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (t0 + q * stride < n) {
                w[t0 + q * stride] = v[q];
                acc = fma(v[q], v[q], acc);
            }
    }
    if (!gm_grid_sums(&acc, 1, partial, counter, red, tot)) return;
    if (threadIdx.x == 0) {
        const double wn = sqrt(tot[0]);
        if (pass == 0) {
            st->need_reorth = wn < 0.7 * sqrt(st->wb2) ? 1 : 0;
        } else {
            for (int j = 0; j <= i; j++) st->hcol[j] += st->corr[j];
            st->need_reorth = 0;
        }
        st->wn = wn;
    }
}

// Column i: h_{i+1,i} = ||w||, previous rotations, a new rotation, g, the
// residual estimate |g_{i+1}| / ||b||, the history ring, stop tests.
__global__ void k_gm_givens(GmState* st, double* ring, int ring_cap, int i, int m, int max_iter) {
    // the column, the previous rotations and the scalars are loaded by the
    // whole warp at once into shared memory; one thread then runs the serial
    // recurrence there instead of on a chain of dependent global loads
    __shared__ double Rc[GM_MAX_RESTART + 2], cs[GM_MAX_RESTART], sn[GM_MAX_RESTART];
    __shared__ int stop;
    if (threadIdx.x == 0) stop = st->stop;
    for (int r = threadIdx.x; r <= i; r += blockDim.x) Rc[r] = st->hcol[r];
    for (int r = threadIdx.x; r < i; r += blockDim.x) {
        cs[r] = st->cs[r];
        sn[r] = st->sn[r];
    }
    __syncthreads();
    if (threadIdx.x != 0 || stop) return;
    const double hn = st->wn, gi = st->g[i], nb = st->nb, tol = st->tol;
    const int j = st->j, hpos = st->hpos, hlen = st->hlen;
    const int ld = m + 1;
    double* Rg = st->R + (size_t)i * ld;
    Rc[i + 1] = hn;
    st->scale[i + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int r = 0; r < i; r++) {
        const double a = Rc[r], b = Rc[r + 1];
        Rc[r] = cs[r] * a + sn[r] * b;
        Rc[r + 1] = -sn[r] * a + cs[r] * b;
    }
    const double den = hypot(Rc[i], Rc[i + 1]);
    if (!(den > 0.0) || !isfinite(den)) {
        for (int r = 0; r <= i + 1; r++) Rg[r] = Rc[r];
        st->lucky = 2;  // singular: cannot extend the least-squares problem
        st->stop = 1;
        st->i_done = i;
        return;
    }
    const double c = Rc[i] / den, sv = Rc[i + 1] / den;
    st->cs[i] = c;
    st->sn[i] = sv;
    Rc[i] = den;
    Rc[i + 1] = 0.0;
    for (int r = 0; r <= i + 1; r++) Rg[r] = Rc[r];
    const double g1 = -sv * gi;
    st->g[i + 1] = g1;
    st->g[i] = c * gi;
    st->j = j + 1;
    const double res = fabs(g1) / nb;
    st->res = res;
    ring[hpos] = res;
    st->hpos = (hpos + 1) % ring_cap;
    if (hlen < ring_cap) st->hlen = hlen + 1;
    st->i_done = i + 1;
    if (hn == 0.0) st->lucky = 1;
    if (!(res >= tol) || hn == 0.0 || j + 1 >= max_iter || !isfinite(res)) st->stop = 1;
}

// y = R^{-1} g (back substitution, i_done columns).
__global__ void k_gm_solve(GmState* st, int m) {
    if (threadIdx.x != 0) return;
    const int ld = m + 1, ni = st->i_done;
    for (int r = ni - 1; r >= 0; r--) {
        double s = st->g[r];
        for (int c = r + 1; c < ni; c++) s -= st->R[(size_t)c * ld + r] * st->y[c];
        st->y[r] = s / st->R[(size_t)r * ld + r];
    }
}

// x += sum_j y_j scale_j V_j.
__global__ void __launch_bounds__(256) k_gm_xupdate(const GmState* st, const double* __restrict__ V, double* x,
                                                     int64_t n) {
    __shared__ double coef[GM_MAX_RESTART];
    const int ni = st->i_done;
    for (int j = threadIdx.x; j < ni; j += blockDim.x) coef[j] = st->y[j] * st->scale[j];
    __syncthreads();
    if (ni == 0) return;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double v = x[t];
        for (int j = 0; j < ni; j++) v = fma(coef[j], V[(size_t)j * n + t], v);
        x[t] = v;
    }
}

// Eqs. 3-6 over the ring, one block.
__global__ void k_gm_metrics(GmState* st, const double* ring, int t) {
    __shared__ double red[32];
    const int cap = t + 1, hpos = st->hpos;
    double s = 0.0;
    for (int i = threadIdx.x; i < t; i += blockDim.x) s += ring[(hpos + i) % cap];
    s = block_sum(s, red);
    __shared__ double avg_sh;
    if (threadIdx.x == 0) avg_sh = s / t;
    __syncthreads();
    const double avg = avg_sh;
    double v = 0.0, nd = 0.0;
    for (int i = threadIdx.x; i < t; i += blockDim.x) {
        const double a = ring[(hpos + i) % cap], b = ring[(hpos + i + 1) % cap];
        v += (a - avg) * (a - avg);
        nd += a > b ? 1.0 : 0.0;
    }
    v = block_sum(v, red);
    nd = block_sum(nd, red);
    if (threadIdx.x == 0) {
        st->rsd = sqrt(v / t) / avg;
        st->ndec = nd;
        const double first = ring[hpos % cap], prev = ring[(hpos + t - 1) % cap];
        st->reldec = (first - prev) / first;
    }
}

}  // namespace gse

using namespace gse;

// The GMRES workspace of a handle: the basis V ((restart + 1) n doubles),
// reduction partials, counters, the residual ring and the device state, kept
// in the handle (pooled device memory) from its first GMRES solve on, so a
// solve allocates nothing once a handle has run one of the same or a larger
// restart length.  gse_free returns it to the pool.
struct GmWork {
    double* V = nullptr;
    double* partial = nullptr;
    unsigned* counter = nullptr;
    double* ring = nullptr;
    GmState* st = nullptr;
    GmState* hst = nullptr;
};

static int gm_workspace(gse_matrix* h, int m, int nblk, cudaStream_t s, GmWork* w) {
    if (!h->ws) h->ws = new Workspace();
    Workspace* W = h->ws;
    const int64_t n = h->v.n_rows;
    if (!W->V || W->V_cols < m + 1) {
        if (W->V) {
            cudaStreamSynchronize(s);
            h->bytes_ws -= (size_t)W->V_cols * (size_t)(n + 2) * sizeof(double);
            pool_free(W->V);
            W->V = nullptr;
            W->V_cols = 0;
        }
        if (pool_alloc(&W->V, (size_t)(m + 1) * (size_t)(n + 2), &h->bytes_ws, s) != GSE_OK) return GSE_ERR_OOM;
        W->V_cols = m + 1;
    }
    const size_t scratch = (size_t)(GM_MAX_RESTART + 2) * (size_t)nblk + GM_RING_MAX + 2 * (sizeof(GmState) / 8 + 1) + 8;
    if (!W->gm_scratch || W->gm_scratch_n < scratch) {
        if (W->gm_scratch) {
            cudaStreamSynchronize(s);
            h->bytes_ws -= W->gm_scratch_n * sizeof(double);
            pool_free(W->gm_scratch);
            W->gm_scratch = nullptr;
            W->gm_scratch_n = 0;
        }
        if (pool_alloc(&W->gm_scratch, scratch, &h->bytes_ws, s) != GSE_OK) return GSE_ERR_OOM;
        W->gm_scratch_n = scratch;
    }
    if (!W->gm_host && cudaMallocHost(&W->gm_host, sizeof(GmState)) != cudaSuccess) {
        cudaGetLastError();
        W->gm_host = nullptr;
        return GSE_ERR_OOM;
    }
    double* p = W->gm_scratch;
    w->V = W->V;
    w->partial = p;
    p += (size_t)(GM_MAX_RESTART + 2) * (size_t)nblk;
    w->ring = p;
    p += GM_RING_MAX;
    w->st = reinterpret_cast<GmState*>(p);
    p += sizeof(GmState) / 8 + 1;
    w->counter = reinterpret_cast<unsigned*>(p);
    w->hst = static_cast<GmState*>(W->gm_host);
    return GSE_OK;
}

static bool level_ok_gm(const gse_matrix* h, int k) { return level_available(h, k); }

extern "C" int gse_gmres(gse_handle h, const double* b, double* x, double tol, const gse_step_policy* pol,
                         gse_solve_info* info, void* stream) {
    if (!h || !b || !x || !pol || !(tol > 0)) return GSE_ERR_INVALID;
    const int m = pol->restart;
    if (m < 1 || m > GM_MAX_RESTART || pol->t < 1 || pol->t > GM_RING_MAX - 1 || pol->max_iter < 1)
        return GSE_ERR_INVALID;
    if (!level_ok_gm(h, pol->k_start) || !level_ok_gm(h, pol->k_max)) return GSE_ERR_INVALID;
    const bool base = pol->k_start > 3 || pol->k_max > 3;
    if (base && pol->k_start != pol->k_max) return GSE_ERR_INVALID;
    if (!base && pol->k_start > pol->k_max) return GSE_ERR_INVALID;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->v.n_rows;
    GmWork w;
    int nblk = h->num_sms * 4;
    const int64_t need = (n + 255) / 256;
    if (nblk > need) nblk = (int)(need < 1 ? 1 : need);
    const int wrc = gm_workspace(h, m, nblk, s, &w);
    if (wrc != GSE_OK) return wrc;
    cudaMemsetAsync(w.counter, 0, 4 * sizeof(unsigned), s);
    cudaMemsetAsync(h->d_err, 0, sizeof(int), s);   // this solve's bounded-wait record starts clear
    memset(w.hst, 0, sizeof(GmState));
    w.hst->tol = tol;
    w.hst->nb = 1.0;
    cudaMemcpyAsync(w.st, w.hst, sizeof(GmState), cudaMemcpyHostToDevice, s);
    // ||b||
    k_gm_norm<<<nblk, 256, 0, s>>>(w.st, b, n, w.partial, w.counter);
    cudaMemcpyAsync(w.hst, w.st, sizeof(GmState), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    const double nb = sqrt(w.hst->wb2);
    int k = pol->k_start, status = GSE_MAXITER, j = 0;
    int sw[3] = {-1, -1, -1};
    if (!base) sw[k - 1] = 0;
    double res = 0.0, true_res = 0.0;
    const int ring_cap = pol->t + 1;
    double* V = w.V;
    auto true_residual = [&](int level) -> double {
        SpmvArgs a = {};
        a.x = x;
        a.y = V;
        a.b = b;
        launch_spmv(h, level, EPI_RESID, a, s);
        k_gm_norm<<<nblk, 256, 0, s>>>(w.st, V, n, w.partial, w.counter);
        cudaMemcpyAsync(w.hst, w.st, sizeof(GmState), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        return sqrt(w.hst->wb2) / nb;
    };
    if (!(nb > 0.0)) {
        cudaMemsetAsync(x, 0, n * sizeof(double), s);
        status = isfinite(nb) ? GSE_OK : GSE_NONFINITE;
    } else {
        // device state for the cycles
        w.hst->nb = nb;
        w.hst->j = 0;
        w.hst->hlen = 0;
        w.hst->hpos = 0;
        cudaMemcpyAsync(w.st, w.hst, sizeof(GmState), cudaMemcpyHostToDevice, s);
        bool v0_ready = false;
        while (true) {
            const int j_before = j;
            if (!v0_ready) {
                SpmvArgs a = {};
                a.x = x;
                a.y = V;
                a.b = b;
                launch_spmv(h, k, EPI_RESID, a, s);
            }
            v0_ready = false;
            k_gm_start<<<nblk, 256, 0, s>>>(w.st, V, n, w.partial, w.counter);
            for (int i = 0; i < m; i++) {
                SpmvArgs a = {};
                a.x = V + (size_t)i * n;
                a.y = V + (size_t)(i + 1) * n;
                a.skip_flag = &w.st->stop;
                launch_spmv(h, k, EPI_STORE, a, s);
                k_gm_dots<<<nblk, 256, 0, s>>>(w.st, V, n, i, 0, w.partial, w.counter);
                k_gm_axpy<<<nblk, 256, 0, s>>>(w.st, V, n, i, 0, w.partial, w.counter);
                k_gm_dots<<<nblk, 256, 0, s>>>(w.st, V, n, i, 1, w.partial, w.counter);
                k_gm_axpy<<<nblk, 256, 0, s>>>(w.st, V, n, i, 1, w.partial, w.counter);
                k_gm_givens<<<1, 32, 0, s>>>(w.st, w.ring, ring_cap, i, m, pol->max_iter);
            }
            k_gm_solve<<<1, 32, 0, s>>>(w.st, m);
            k_gm_xupdate<<<nblk, 256, 0, s>>>(w.st, V, x, n);
            cudaMemcpyAsync(w.hst, w.st, sizeof(GmState), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) { status = GSE_ERR_CUDA; break; }
            j = w.hst->j;
            res = w.hst->res;
            if (!isfinite(res)) { status = GSE_NONFINITE; break; }
            bool step = false, restart_same = false;
            if (res < tol) {
                true_res = true_residual(pol->k_max);
                if (true_res < tol) { status = GSE_OK; break; }
                if (k < pol->k_max) step = true;
                else { v0_ready = true; restart_same = true; }   // V[0] already holds b - A_kmax x
            } else if (w.hst->lucky == 2) {
                if (k < pol->k_max) step = true;
                else { status = GSE_BREAKDOWN; break; }
            }
            if (j >= pol->max_iter) { status = GSE_MAXITER; break; }
            if (!step && !restart_same && !base && k < pol->k_max && !(pol->flags & GSE_POLICY_NO_STAGNATION) &&
                pol->m > 0 && j >= pol->l && j / pol->m > j_before / pol->m && w.hst->hlen >= ring_cap) {
                k_gm_metrics<<<1, 256, 0, s>>>(w.st, w.ring, pol->t);
                cudaMemcpyAsync(w.hst, w.st, sizeof(GmState), cudaMemcpyDeviceToHost, s);
                cudaStreamSynchronize(s);
                const double thr = pol->ndec_limit > 0 ? (double)pol->ndec_limit : 0.5 * pol->t;
                const double rsd = w.hst->rsd, nd = w.hst->ndec, rd = w.hst->reldec;
                if ((rsd > pol->rsd_limit && nd < thr) || (nd >= thr && rd < pol->reldec_limit) || nd == 0.0)
                    step = true;
            }
            if (step) {
                k++;
                sw[k - 1] = j;
                // clear the history
                GmState* hs = w.hst;
                hs->hlen = 0;
                hs->hpos = 0;
                cudaMemcpyAsync(&w.st->hlen, &hs->hlen, 2 * sizeof(int), cudaMemcpyHostToDevice, s);
                if (k == pol->k_max && res < tol) v0_ready = true;   // V[0] = b - A_kmax x already
            }
        }
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->status = status;
        info->iters = j;
        info->k_final = base ? 0 : k;
        for (int i = 0; i < 3; i++) info->switch_iter[i] = base ? -1 : sw[i];
        info->rel_res_rec = res;
        info->rel_res_true = nb > 0.0 ? true_residual(pol->k_max) : 0.0;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    cudaStreamSynchronize(s);
    int err = 0;
    cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err && status != GSE_ERR_CUDA) {
        status = GSE_TIMEOUT;   // a bounded device-side wait gave up
        if (info) info->status = status;
    }
    if (status == GSE_ERR_CUDA) return status;
    return cudaGetLastError() == cudaSuccess ? status : GSE_ERR_CUDA;
}
