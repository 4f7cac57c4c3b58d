// msim_api.cu -- C ABI of the batched muscle-driven forward-dynamics library (include/msim.h).
//
// Host side only: validates model descriptions, builds the flat device images (image.h),
// owns the state buffers and launches the kernels of step_kernels.cu.  No dynamics arithmetic
// runs on the host: even the reference muscle lengths L0 = L(q = 0) are computed by the device
// kernel at create time.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/msim.h"
#include "gemm_tc.h"
#include "mlp.h"
#include "image.h"
#include "surrogate.h"
#include "handle.h"
#include "kernels.h"

using namespace msim;

namespace {

thread_local std::string g_create_error;

int pad4(int x) { return (x + 3) & ~3; }
size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

bool finite_all(const float* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

#define FAIL(...)                                            \
    do {                                                     \
        char buf_[256];                                      \
        std::snprintf(buf_, sizeof(buf_), __VA_ARGS__);      \
        err = buf_;                                          \
        return false;                                        \
    } while (0)

bool build_image(const msim_model_desc& d, ModelHost& out, std::string& err) {
    const int nb = d.n_bodies, n = d.n_dofs, m = d.n_muscles, np = d.n_points, ns = d.n_spheres;
    if (nb < 1 || nb > 255) FAIL("n_bodies must be in [1, 255] (got %d)", nb);
    if (n < 1 || n > 255) FAIL("n_dofs must be in [1, 255] (got %d)", n);
    if (m < 0 || m > 4096) FAIL("n_muscles must be in [0, 4096] (got %d)", m);
    if (ns < 0 || ns > kMaxSpheres) FAIL("n_spheres must be in [0, %d] (got %d)", kMaxSpheres, ns);
    if (np < 0 || np < 2 * m) FAIL("n_points must be >= 2 n_muscles");
    if (!d.body_parent || !d.body_ndof || !d.body_offset || !d.body_mass || !d.body_com || !d.body_inertia ||
        !d.dof_axis)
        FAIL("missing body or DoF array");
    if (m > 0 && (!d.muscle_point_start || !d.muscle_fmax || !d.muscle_lopt || !d.point_body || !d.point_pos))
        FAIL("missing muscle array");
    if (ns > 0 && (!d.sphere_body || !d.sphere_pos || !d.sphere_radius)) FAIL("missing sphere array");
    if (!finite_all(d.body_offset, 3 * nb) || !finite_all(d.body_mass, nb) || !finite_all(d.body_com, 3 * nb) ||
        !finite_all(d.body_inertia, 6 * nb) || !finite_all(d.dof_axis, 3 * n))
        FAIL("non-finite body or DoF parameter");
    if (!(d.limit_delta >= 0.f) || !std::isfinite(d.limit_delta)) FAIL("limit_delta must be finite and >= 0");

    // ---- DoF tree
    std::vector<int> dof0(nb), dof_body(n), dpar(n), depth(n), bdepth(nb);
    int acc = 0;
    for (int b = 0; b < nb; ++b) {
        const int pb = d.body_parent[b];
        if (pb < -1 || pb >= b) FAIL("body_parent[%d] = %d must be in [-1, %d)", b, pb, b);
        const int k = d.body_ndof[b];
        if (d.free_root && b == 0) {
            if (pb != -1 || k != 6) FAIL("free root: body 0 must be a root with 6 DoFs");
        } else if (k < 1 || k > 3) {
            FAIL("body_ndof[%d] = %d must be 1..3", b, k);
        }
        dof0[b] = acc;
        for (int j = 0; j < k; ++j) {
            const int dd = acc + j;
            dof_body[dd] = b;
            dpar[dd] = (j > 0) ? dd - 1 : (pb < 0 ? -1 : dof0[pb] + d.body_ndof[pb] - 1);
            depth[dd] = dpar[dd] < 0 ? 0 : depth[dpar[dd]] + 1;
            if (depth[dd] > kMaxDepth) FAIL("DoF depth above %d", kMaxDepth);
        }
        acc += k;
        bdepth[b] = pb < 0 ? 0 : bdepth[pb] + 1;
    }
    if (acc != n) FAIL("sum of body_ndof (%d) != n_dofs (%d)", acc, n);
    if (d.free_root != 0 && d.free_root != 1) FAIL("free_root must be 0 or 1");
    for (int i = d.free_root ? 6 : 0; i < n; ++i) {   // the free root's axes are implied
        const float* a = d.dof_axis + 3 * i;
        const double nrm = std::sqrt(double(a[0]) * a[0] + double(a[1]) * a[1] + double(a[2]) * a[2]);
        if (std::fabs(nrm - 1.0) > 1e-4) FAIL("dof_axis[%d] is not a unit vector", i);
    }
    std::vector<int> row(n);
    int nM = 0, max_depth = 0;
    for (int i = 0; i < n; ++i) {
        row[i] = nM;
        nM += depth[i] + 1;
        max_depth = std::max(max_depth, depth[i]);
    }
    std::vector<uint8_t> anc(nM);
    std::vector<uint16_t> rowanc(nM);   // packed row start of the ancestor of each entry
    for (int i = 0; i < n; ++i)
        for (int a = i; a >= 0; a = dpar[a]) {
            anc[row[i] + depth[a]] = (uint8_t)a;
            rowanc[row[i] + depth[a]] = (uint16_t)row[a];
        }
    if (nM > 65535) FAIL("packed mass matrix above 65535 entries");

    // body levels and children
    const int n_bl = *std::max_element(bdepth.begin(), bdepth.end()) + 1;
    std::vector<uint8_t> border;
    std::vector<int16_t> blevel(n_bl + 1, 0);
    for (int l = 0; l < n_bl; ++l) {
        blevel[l] = (int16_t)border.size();
        for (int b = 0; b < nb; ++b)
            if (bdepth[b] == l) border.push_back((uint8_t)b);
    }
    blevel[n_bl] = (int16_t)border.size();
    std::vector<uint8_t> child;
    std::vector<int> child0(nb), nchild(nb);
    for (int b = 0; b < nb; ++b) {
        child0[b] = (int)child.size();
        for (int c = b + 1; c < nb; ++c)
            if (d.body_parent[c] == b) child.push_back((uint8_t)c);
        nchild[b] = (int)child.size() - child0[b];
    }
    // body chains for the subtree sums: maximal runs of single-child bodies, bottom to top, in
    // rounds (a chain whose bottom has children comes after the chains hanging below it)
    std::vector<int16_t> cround, cstart;
    std::vector<uint8_t> cbody;
    {
        std::vector<std::vector<int>> chains;
        std::vector<int> top_of(nb, -1);
        for (int t = 0; t < nb; ++t) {
            const int pb = d.body_parent[t];
            if (pb >= 0 && nchild[pb] == 1) continue;   // not a chain top
            std::vector<int> path{t};
            while (nchild[path.back()] == 1) path.push_back(child[child0[path.back()]]);
            std::reverse(path.begin(), path.end());
            top_of[t] = (int)chains.size();
            chains.push_back(path);
        }
        std::vector<int> rnd(chains.size(), -1);
        // bodies are numbered parents first, so chains whose top has the larger index are deeper:
        // resolve rounds from the last chain top backwards
        std::vector<int> order(chains.size());
        for (size_t c = 0; c < chains.size(); ++c) order[c] = (int)c;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return chains[a].back() > chains[b].back(); });
        for (int c : order) {
            const int bot = chains[c][0];
            int r = 0;
            for (int k = 0; k < nchild[bot]; ++k) r = std::max(r, 1 + rnd[top_of[child[child0[bot] + k]]]);
            rnd[c] = r;
        }
        const int nr = chains.empty() ? 0 : *std::max_element(rnd.begin(), rnd.end()) + 1;
        for (int r = 0; r < nr; ++r) {
            cround.push_back((int16_t)(cstart.size()));
            for (size_t c = 0; c < chains.size(); ++c)
                if (rnd[c] == r) {
                    cstart.push_back((int16_t)cbody.size());
                    for (int b : chains[c]) cbody.push_back((uint8_t)b);
                }
        }
        cround.push_back((int16_t)cstart.size());
        cstart.push_back((int16_t)cbody.size());
    }
    // DoF levels; each node of the factorisation as one word (node_dof / node_depth / node_row
    // in image.h), so that its lanes need one shared-memory load per node, not two dependent ones
    const int n_dl = max_depth + 1;
    std::vector<uint32_t> dorder;
    std::vector<int16_t> dlevel(n_dl + 1, 0);
    for (int l = 0; l < n_dl; ++l) {
        dlevel[l] = (int16_t)dorder.size();
        for (int i = 0; i < n; ++i)
            if (depth[i] == l) dorder.push_back((uint32_t)i | ((uint32_t)depth[i] << 8) | ((uint32_t)row[i] << 16));
    }
    dlevel[n_dl] = (int16_t)dorder.size();
    // CRBA work order: DoFs by decreasing packed-row length; the kernel deals them to however
    // many lanes a group has in a snake (0..N-1, N-1..0, ...), so that every lane gets a similar
    // number of entries.  Entry t: DoF | body << 8 | depth << 16, then its packed row start (one
    // 8-byte load per lane instead of a lookup of the DoF record).
    std::vector<int> byrow(n);
    for (int i = 0; i < n; ++i) byrow[i] = i;
    std::stable_sort(byrow.begin(), byrow.end(), [&](int a, int b) { return depth[a] > depth[b]; });
    std::vector<uint32_t> crba_order(2 * n);
    for (int t = 0; t < n; ++t) {
        const int dd = byrow[t];
        crba_order[2 * t] = (uint32_t)dd | ((uint32_t)dof_body[dd] << 8) | ((uint32_t)depth[dd] << 16);
        crba_order[2 * t + 1] = (uint32_t)row[dd];
    }
    // pair table: p -> (ia, ib), ib <= ia, row by row
    std::vector<uint16_t> tri;
    for (int ia = 0; ia <= max_depth; ++ia)
        for (int ib = 0; ib <= ia; ++ib) tri.push_back((uint16_t)(ia | (ib << 8)));

    // ---- muscles
    std::vector<MuscleRec> mus(m);
    std::vector<PointRec> pts(np);
    // wrapping cylinders
    const int nw = d.n_wraps;
    if (nw < 0 || nw > 255) FAIL("n_wraps must be 0..255");
    if (nw > 0 && (!d.wrap_muscle || !d.wrap_segment || !d.wrap_body || !d.wrap_center || !d.wrap_axis ||
                   !d.wrap_radius))
        FAIL("wrap arrays are NULL");
    std::vector<int> wrap_of(m, -1);
    for (int w = 0; w < nw; ++w) {
        const int k = d.wrap_muscle[w];
        if (k < 0 || k >= m) FAIL("wrap %d: muscle out of range", w);
        if (wrap_of[k] >= 0) FAIL("muscle %d has two wrapping surfaces", k);
        wrap_of[k] = w;
        const int kind = d.wrap_kind ? d.wrap_kind[w] : 0;
        if (kind != 0 && kind != 1) FAIL("wrap %d: kind must be 0 (cylinder) or 1 (sphere)", w);
        if (!(d.wrap_radius[w] > 0.f) || !finite_all(d.wrap_center + 3 * w, 3))
            FAIL("wrap %d: radius must be > 0 and centre finite", w);
        if (kind == 0) {
            const float* ax = d.wrap_axis + 3 * w;
            if (!finite_all(ax, 3) || !(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2] > 1e-12f))
                FAIL("wrap %d: cylinder axis must be finite and non-zero", w);
        }
    }
    std::vector<WrapRec> wraps(nw);
    // compliant tendons
    int n_ten = 0;
    if (d.muscle_tendon_strain)
        for (int k = 0; k < m; ++k) {
            const float t = d.muscle_tendon_strain[k];
            if (!(t >= 0.f && t <= 0.5f)) FAIL("muscle %d: tendon strain at F_max must be 0 (rigid) or in (0, 0.5]", k);
            n_ten += t > 0.f;
        }
    auto compliant = [&](int k) { return d.muscle_tendon_strain && d.muscle_tendon_strain[k] > 0.f; };
    std::vector<uint32_t> cross;
    std::vector<int32_t> mus_ptr(m + 1, 0), mus_dof, mus_body;
    std::vector<uint8_t> one_joint(m, 1);
    if (m > 0) {
        if (d.muscle_point_start[0] != 0 || d.muscle_point_start[m] != np)
            FAIL("muscle_point_start must start at 0 and end at n_points");
        if (!finite_all(d.point_pos, 3 * np) || !finite_all(d.muscle_fmax, m) || !finite_all(d.muscle_lopt, m))
            FAIL("non-finite muscle parameter");
    }
    for (int k = 0; k < m; ++k) {
        const int j0 = d.muscle_point_start[k], j1 = d.muscle_point_start[k + 1];
        const int cnt = j1 - j0;
        if (cnt < 2 || cnt > kMaxPts) FAIL("muscle %d has %d points (allowed 2..%d)", k, cnt, kMaxPts);
        if (!(d.muscle_lopt[k] > 0.f) || !(d.muscle_fmax[k] >= 0.f)) FAIL("muscle %d: l_opt must be > 0", k);
        for (int j = j0; j < j1; ++j)
            if (d.point_body[j] < 0 || d.point_body[j] >= nb) FAIL("point %d: body out of range", j);
        const int A = d.point_body[j0], B = d.point_body[j1 - 1];
        std::vector<int> chain;   // bodies strictly below A down to B, root to leaf
        int b = B;
        while (b != A && b >= 0) {
            chain.push_back(b);
            b = d.body_parent[b];
        }
        if (b != A) FAIL("muscle %d: insertion body is not a descendant of the origin body", k);
        std::reverse(chain.begin(), chain.end());
        auto pos_of = [&](int body) -> int {
            if (body == A) return 0;
            for (size_t t = 0; t < chain.size(); ++t)
                if (chain[t] == body) return (int)t + 1;
            return -1;
        };
        std::vector<int> ccount(chain.size() + 1, 0);
        for (size_t t = 0; t < chain.size(); ++t) ccount[t + 1] = ccount[t] + d.body_ndof[chain[t]];
        const int nx = ccount.back();
        if (nx > kMaxCross) FAIL("muscle %d crosses %d DoFs (max %d)", k, nx, kMaxCross);
        int prev = 0;
        for (int j = j0; j < j1; ++j) {
            const int t = pos_of(d.point_body[j]);
            if (t < 0 || t < prev) FAIL("muscle %d: path points must follow the origin-to-insertion chain", k);
            if (j > j0 && t - prev > 1) one_joint[k] = 0;   // this segment spans several joints
            prev = t;
            PointRec& P = pts[j];
            P.pos[0] = d.point_pos[3 * j]; P.pos[1] = d.point_pos[3 * j + 1]; P.pos[2] = d.point_pos[3 * j + 2];
            P.body_cross = d.point_body[j] | (ccount[t] << 8);
        }
        MuscleRec& M = mus[k];
        std::memset(&M, 0, sizeof(M));
        if (wrap_of[k] >= 0) {
            const int w = wrap_of[k], seg = d.wrap_segment[w], bw = d.wrap_body[w];
            if (seg < 1 || seg >= cnt) FAIL("wrap %d: segment must be 1..points-1 of muscle %d", w, k);
            const int tw = (bw >= 0 && bw < nb) ? pos_of(bw) : -1;
            if (tw < pos_of(d.point_body[j0 + seg - 1]) || tw > pos_of(d.point_body[j0 + seg]))
                FAIL("wrap %d: body must lie on the chain between the wrapped segment's bodies", w);
            WrapRec& W = wraps[w];
            const int kind = d.wrap_kind ? d.wrap_kind[w] : 0;
            const float* ax = d.wrap_axis + 3 * w;
            const float an = kind ? 1.f : std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
            for (int c = 0; c < 3; ++c) {
                W.center[c] = d.wrap_center[3 * w + c];
                W.axis[c] = kind ? 0.f : ax[c] / an;
            }
            W.radius = d.wrap_radius[w];
            W.body_cross = bw | (ccount[tw] << 8) | (seg << 16) | (kind << 24);
            M.wrap = (uint8_t)(w + 1);
        }
        M.fmax = d.muscle_fmax[k];
        M.inv_lopt = 1.f / d.muscle_lopt[k];
        M.L0 = 0.f;
        M.inv_vmax = 1.f / (d.vmax_per_lopt * d.muscle_lopt[k]);
        M.p0 = j0;
        M.x0 = (int32_t)cross.size();
        M.np = (uint8_t)cnt;
        M.nx = (uint8_t)nx;
        M.dep0 = nx > 0 ? (uint8_t)depth[dof0[chain[0]]] : 0;
        M.orig = k;
        for (size_t t = 0; t < chain.size(); ++t)
            for (int j = 0; j < d.body_ndof[chain[t]]; ++j) {
                const int dd = dof0[chain[t]] + j;
                cross.push_back((uint32_t)dd | ((uint32_t)chain[t] << 8) | ((uint32_t)row[dd] << 16));
                mus_dof.push_back(dd);
                mus_body.push_back(chain[t]);
            }
        mus_ptr[k + 1] = (int32_t)cross.size();
    }
    // records sorted by (compliant tendon, wrapped segment, points, crossed DoFs): a warp's 32
    // lanes then share loop trip counts and take the tendon and wrapping branches together;
    // then by the bodies of the path points in order, so that lanes reading point j's body frame
    // often read the same one (a broadcast instead of a bank conflict)
    std::vector<int> wseg(m, 0);
    for (int k = 0; k < m; ++k)
        if (mus[k].wrap) wseg[k] = d.wrap_segment[mus[k].wrap - 1];
    {
        std::vector<int> order(m);
        for (int k = 0; k < m; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const MuscleRec &A = mus[a], &B = mus[b];
            if (compliant(A.orig) != compliant(B.orig)) return compliant(B.orig);
            if (wseg[a] != wseg[b]) return wseg[a] < wseg[b];
            if (A.np != B.np) return A.np < B.np;
            if (A.nx != B.nx) return A.nx < B.nx;
            const int* pa = d.point_body + d.muscle_point_start[A.orig];
            const int* pb = d.point_body + d.muscle_point_start[B.orig];
            for (int j = 0; j < A.np; ++j)
                if (pa[j] != pb[j]) return pa[j] < pb[j];
            return false;
        });
        std::vector<MuscleRec> sorted(m);
        for (int k = 0; k < m; ++k) sorted[k] = mus[order[k]];
        mus.swap(sorted);
    }
    // via points interleaved by groups of 32 muscle records (the muscles one warp handles in one
    // pass): point j of record r at group base + 32 j + r % 32, so that a warp's loads of point j
    // are one contiguous run
    int np_lay = 0;
    {
        std::vector<PointRec> lay;
        for (int g0 = 0; g0 < m; g0 += 32) {
            int npg = 0;
            for (int r = g0; r < std::min(m, g0 + 32); ++r) npg = std::max(npg, (int)mus[r].np);
            const int base = (int)lay.size();
            lay.resize(base + 32 * npg);
            for (int r = g0; r < std::min(m, g0 + 32); ++r) {
                const int src = mus[r].p0;
                for (int j = 0; j < mus[r].np; ++j) lay[base + 32 * j + (r - g0)] = pts[src + j];
                mus[r].p0 = base + (r - g0);
            }
        }
        pts.swap(lay);
        np_lay = (int)pts.size();
    }
    std::vector<TendonRec> tens(n_ten ? m : 0);
    for (int r = 0; r < (int)tens.size(); ++r) {
        const int k = mus[r].orig;
        tens[r].inv_eps0 = compliant(k) ? 1.f / d.muscle_tendon_strain[k] : 0.f;
        tens[r].lopt = d.muscle_lopt[k];
        tens[r].vmax = d.vmax_per_lopt * d.muscle_lopt[k];
        tens[r].pad = 0.f;
    }
    if (!(d.vmax_per_lopt > 0.f) || !(d.tau_act > 0.f) || !(d.tau_deact > 0.f)) FAIL("time constants must be > 0");

    // ---- spheres
    std::vector<SphereRec> sph(ns);
    for (int i = 0; i < ns; ++i) {
        const int b = d.sphere_body[i];
        if (b < 0 || b >= nb) FAIL("sphere %d: body out of range", i);
        std::memset(&sph[i], 0, sizeof(SphereRec));
        for (int c = 0; c < 3; ++c) sph[i].pos[c] = d.sphere_pos[3 * i + c];
        sph[i].radius = d.sphere_radius[i];
        sph[i].body = b;
        sph[i].last_dof = dof0[b] + d.body_ndof[b] - 1;
    }

    // ---- records
    std::vector<BodyRec> bodies(nb);
    for (int b = 0; b < nb; ++b) {
        BodyRec& B = bodies[b];
        std::memset(&B, 0, sizeof(B));
        for (int c = 0; c < 3; ++c) { B.off[c] = d.body_offset[3 * b + c]; B.com[c] = d.body_com[3 * b + c]; }
        B.mass = d.body_mass[b];
        B.parent = d.body_parent[b];
        for (int c = 0; c < 6; ++c) B.I[c] = d.body_inertia[6 * b + c];
        B.dof0 = (int16_t)dof0[b];
        B.ndof = (int16_t)d.body_ndof[b];
        B.child0 = (int16_t)child0[b];
        B.nchild = (int16_t)nchild[b];
    }
    std::vector<DofRec> dofs(n);
    for (int i = 0; i < n; ++i) {
        DofRec& D = dofs[i];
        std::memset(&D, 0, sizeof(D));
        for (int c = 0; c < 3; ++c) D.axis[c] = d.dof_axis[3 * i + c];
        D.lo = d.dof_limit ? d.dof_limit[2 * i] : 0.f;
        D.hi = d.dof_limit ? d.dof_limit[2 * i + 1] : 0.f;
        D.damp = d.dof_damping ? d.dof_damping[i] : 0.f;
        if (d.free_root && i < 6) {   // world axes x, y, z (translations, then rotations)
            for (int c = 0; c < 3; ++c) D.axis[c] = (c == i % 3) ? 1.f : 0.f;
            if (D.lo < D.hi) FAIL("free root: DoF %d must have no limit", i);
        }
        D.row = row[i];
        D.parent = (int16_t)dpar[i];
        D.depth = (uint8_t)depth[i];
        D.body = (uint8_t)dof_body[i];
    }

    // ---- header and blob
    ImgHeader& h = out.hdr;
    std::memset(&h, 0, sizeof(h));
    h.n = n; h.m = m; h.nb = nb; h.np = np; h.ns = ns;
    h.n_packed = nM;
    h.nnz = (int32_t)cross.size();
    h.n_blevels = n_bl;
    h.n_dlevels = n_dl;
    h.max_depth = max_depth;
    h.n_tri = (int32_t)tri.size();
    size_t off = align16(sizeof(ImgHeader));
    auto place = [&](size_t bytes) {
        const size_t o = off;
        off = align16(off + bytes);
        return (int32_t)o;
    };
    h.o_body = place(sizeof(BodyRec) * nb);
    h.o_dof = place(sizeof(DofRec) * n);
    h.o_sphere = place(sizeof(SphereRec) * ns);
    h.o_border = place(border.size());
    h.o_blevel = place(sizeof(int16_t) * blevel.size());
    h.o_child = place(child.size());
    h.o_anc = place(anc.size());
    h.o_dorder = place(sizeof(uint32_t) * dorder.size());
    h.o_dlevel = place(sizeof(int16_t) * dlevel.size());
    h.n_crounds = (int32_t)cround.size() - 1;
    h.n_chains = (int32_t)cstart.size() - 1;
    h.o_chain = place(sizeof(int16_t) * (cround.size() + cstart.size()) + cbody.size());
    h.o_tri = place(sizeof(uint16_t) * tri.size());
    h.o_rowanc = place(sizeof(uint16_t) * rowanc.size());
    h.o_crba = place(sizeof(uint32_t) * crba_order.size());
    // last: the sections that may stay in global memory (staged_bytes in image.h)
    h.o_muscle = place(sizeof(MuscleRec) * m);
    h.o_cross = place(sizeof(uint32_t) * cross.size());
    h.o_point = place(sizeof(PointRec) * np_lay);
    h.o_wrap = place(sizeof(WrapRec) * std::max(nw, 1));
    h.n_tendons = n_ten;
    h.o_tendon = n_ten ? place(sizeof(TendonRec) * m) : 0;
    h.total_bytes = (int32_t)off;
    // per-environment workspace
    int w = 0;
    auto slot = [&](int floats) {
        const int o = w;
        w += pad4(floats);
        return o;
    };
    h.w_q = slot(n);
    h.w_qd = slot(n);
    h.w_frame = slot(12 * nb);
    h.w_fi = slot(kFiStride * nb);
    h.w_S = slot(6 * n);
    h.w_A = slot(2 * std::max(nM, 12 * nb));
    h.w_v = h.w_A + 6 * nb;    // inside A: velocities and float-float body forces until the mass matrix
    h.w_f = h.w_A + 12 * nb;
    h.w_rhs = slot(n);
    h.w_racc = slot(2 * n);
    h.w_y = h.w_racc;          // the solution replaces the decoded accumulators
    h.w_rk = w;   // last: its size depends on the warps per environment (ws_floats)
    h.w_sph = h.w_rk;          // contact scratch, after the muscles have used the region
    h.max_nx = 1;
    for (int k = 0; k < m; ++k) h.max_nx = std::max(h.max_nx, (int)mus[k].nx);
    for (int c = 0; c < 3; ++c) h.gravity[c] = d.gravity[c];
    h.contact_k = d.contact_k;
    h.contact_c = d.contact_c;
    h.contact_mu = d.contact_mu;
    h.contact_eps2 = d.contact_eps * d.contact_eps;
    h.limit_k = d.limit_k;
    h.limit_c = d.limit_c;
    h.limit_delta = d.limit_delta;
    h.tau_act = d.tau_act;
    h.tau_deact = d.tau_deact;
    const double e4 = std::exp(4.0);
    h.fp_den = (float)(e4 - 1.0);
    h.fp_slope = (float)((4.0 / 0.6) * e4 / (e4 - 1.0));
    h.free_root = d.free_root;
    h.n_wraps = nw;
    const double e3 = std::exp(3.0);
    h.ft_den = (float)(e3 - 4.0);
    h.ft_slope = (float)(3.0 * (e3 - 1.0) / (e3 - 4.0));

    out.blob.assign(h.total_bytes, 0);
    auto put = [&](int32_t o, const void* src, size_t bytes) {
        if (bytes) std::memcpy(out.blob.data() + o, src, bytes);
    };
    put(0, &h, sizeof(h));
    put(h.o_body, bodies.data(), sizeof(BodyRec) * nb);
    put(h.o_dof, dofs.data(), sizeof(DofRec) * n);
    put(h.o_muscle, mus.data(), sizeof(MuscleRec) * m);
    put(h.o_point, pts.data(), sizeof(PointRec) * np_lay);
    if (nw > 0) put(h.o_wrap, wraps.data(), sizeof(WrapRec) * nw);
    if (n_ten) put(h.o_tendon, tens.data(), sizeof(TendonRec) * m);
    put(h.o_sphere, sph.data(), sizeof(SphereRec) * ns);
    put(h.o_cross, cross.data(), sizeof(uint32_t) * cross.size());
    put(h.o_border, border.data(), border.size());
    put(h.o_blevel, blevel.data(), sizeof(int16_t) * blevel.size());
    put(h.o_child, child.data(), child.size());
    put(h.o_anc, anc.data(), anc.size());
    put(h.o_dorder, dorder.data(), sizeof(uint32_t) * dorder.size());
    put(h.o_dlevel, dlevel.data(), sizeof(int16_t) * dlevel.size());
    put(h.o_chain, cround.data(), sizeof(int16_t) * cround.size());
    put(h.o_chain + (int32_t)(sizeof(int16_t) * cround.size()), cstart.data(), sizeof(int16_t) * cstart.size());
    put(h.o_chain + (int32_t)(sizeof(int16_t) * (cround.size() + cstart.size())), cbody.data(), cbody.size());
    put(h.o_tri, tri.data(), sizeof(uint16_t) * tri.size());
    put(h.o_rowanc, rowanc.data(), sizeof(uint16_t) * rowanc.size());
    put(h.o_crba, crba_order.data(), sizeof(uint32_t) * crba_order.size());

    out.dof_parent.assign(dpar.begin(), dpar.end());
    out.dof_depth.assign(depth.begin(), depth.end());
    out.packed_row.assign(row.begin(), row.end());
    out.mus_ptr = mus_ptr;
    out.mus_dof = mus_dof;
    out.mus_body = mus_body;
    out.mus_one_joint_segments = one_joint;
    return true;
}
#undef FAIL

}  // namespace

namespace msim {
void set_global_error(const char* what) { g_create_error = what; }
}  // namespace msim

namespace msim {
namespace host {

msim_status cuda_fail(msim_handle h, cudaError_t e, const char* what) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    if (h) h->err = buf; else g_create_error = buf;
    return (e == cudaErrorMemoryAllocation) ? MSIM_ERR_OOM : MSIM_ERR_CUDA;
}

msim_status arg_fail(msim_handle h, const char* what) {
    if (h) h->err = what; else g_create_error = what;
    return MSIM_ERR_ARG;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int model_grid(msim_handle h, int i) {
    const int ne = h->env_begin[i + 1] - h->env_begin[i];
    const int groups = (ne + h->epb[i] - 1) / h->epb[i];
    const size_t smem = step_smem_bytes(h->models[i].hdr, h->epb[i], h->pts_smem[i], h->wpe[i]);
    const int per_sm =
        std::max(1, step_blocks_per_sm(32 * h->wpe[i] * h->epb[i], smem, h->wpe[i], uses_ext(h->models[i].hdr)));
    return std::max(1, std::min(groups, h->num_sms * per_sm));
}

StepArgs base_args(msim_handle h, int i) {
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.img = h->d_img[i];
    a.wrap = uses_ext(h->models[i].hdr) ? 1 : 0;
    a.stage = h->pts_smem[i];
    a.staged_bytes = staged_bytes(h->models[i].hdr, h->pts_smem[i]);
    a.env_begin = h->env_begin[i];
    a.env_end = h->env_begin[i + 1];
    a.q = h->q; a.qd = h->qd; a.act = h->act; a.eps = h->eps;
    a.pitch_n = h->pitch_n; a.pitch_m = h->pitch_m;
    a.qdd_out = h->qdd; a.force_out = h->force; a.vm_out = h->vm;
    a.env_status = h->env_status; a.gflags = h->gflags;
    a.dt = h->dt;
    a.envs_per_block = h->epb[i];
    a.wpe = h->wpe[i];
    a.timers = h->timers;
    return a;
}

int max_epb(msim_handle h, int i, int stage, int wpe) {
    const ImgHeader& hd = h->models[i].hdr;
    const size_t fixed = step_smem_bytes(hd, 0, stage, wpe);
    const size_t per = (size_t)ws_floats(hd, wpe) * sizeof(float);
    if (fixed + per > h->smem_optin) return 0;
    const int lim = wpe == 1 ? kMaxEnvsPerBlock : std::min(15, 16 / wpe);   // 512 threads, 15 named barriers
    return std::min((int)((h->smem_optin - fixed) / per), lim);
}

// Default launch shape: two warps per environment.  Among the environments per block (<= 8)
// whose resident environments per SM (per block x blocks per SM) reach 85 % of the most any count
// gives (the kernel is latency-bound: throughput follows residency), the one that gives the
// busiest SM the fewest environments, ceil(blocks / block slots) x resident, the larger residency
// on a tie.  Sections are left in global memory (via points, then also the muscle records,
// staging levels 0 and 2) only when that is needed for the chosen count.
void auto_launch(msim_handle h, int i) {
    const int ne = std::max(1, h->env_begin[i + 1] - h->env_begin[i]);
    // one warp per environment for small skeletons (what the autotuner picks for the 30- and
    // 40-DoF bodies), two for larger ones
    const int w = h->models[i].hdr.n <= 48 ? 1 : 2;
    const int emax = w == 1 ? 16 : 8;
    int stage_of[17], per_sm_of[17], cmax = 0;
    for (int e = 1; e <= emax; ++e) {
        stage_of[e] = -1;
        per_sm_of[e] = 0;
        if (e > ne) continue;
        for (int st : {1, 0, 2})
            if (stage_of[e] < 0 && max_epb(h, i, st, w) >= e) stage_of[e] = st;
        if (stage_of[e] < 0) continue;
        const size_t smem = step_smem_bytes(h->models[i].hdr, e, stage_of[e], w);
        per_sm_of[e] = std::max(1, step_blocks_per_sm(32 * w * e, smem, w, uses_ext(h->models[i].hdr)));
        cmax = std::max(cmax, e * per_sm_of[e]);
    }
    int best_e = 1;
    long best_load = -1, best_c = 0;
    for (int e = 1; e <= emax; ++e) {
        if (stage_of[e] < 0) continue;
        const long c = (long)e * per_sm_of[e];
        if (100 * c < 85L * cmax) continue;
        const long blocks = (ne + e - 1) / e;
        const long slots = (long)h->num_sms * per_sm_of[e];
        const long load = (blocks + slots - 1) / slots * c;
        if (best_load < 0 || load < best_load || (load == best_load && c > best_c)) {
            best_load = load;
            best_c = c;
            best_e = e;
        }
    }
    h->wpe[i] = w;
    h->pts_smem[i] = stage_of[best_e] < 0 ? 1 : stage_of[best_e];
    h->epb[i] = best_e;
}

}  // namespace host
}  // namespace msim

using namespace msim::host;

namespace {

// Connectivity of the learned geometry.  Every path segment of the generated models joins points
// on the same or on adjacent bodies, so a segment's length depends on the DoFs of one joint only:
// each muscle length is a sum of one-joint terms, and the moment arm R_kd = -dL_k/dq_d depends on
// the DoFs of d's joint alone.  The network is given that structure: its hidden units are split
// into one block per joint (a body whose DoFs some muscle crosses), a block's first-layer units
// read only that joint's DoFs, the second layer is block diagonal, the length of muscle k reads
// the blocks of the joints k crosses and R_kd the block of d's joint.  The GEMMs stay dense (the
// masked weights are zeros); only training honours the mask.  Block sizes: the hidden width split
// in proportion to sqrt(outputs depending on the joint) x (its DoFs)^2, at least 2 units each: a
// joint's functions have as many arguments as it has DoFs, and a three-angle function takes many
// more units than a one-angle function to the same accuracy (the weights were chosen by the
// moment-arm error of networks trained with several of them).  Returns false (dense network) when
// some segment spans several joints or the width cannot give every joint its 2 units.
bool surrogate_mask(const ModelHost& M, const Mlp* net, int m, std::vector<uint8_t>& mask) {
    for (uint8_t v : M.mus_one_joint_segments)
        if (!v) return false;
    const int nnz = (int)M.mus_dof.size();
    std::map<int, int> block_of;          // joint body -> block index
    std::vector<int> dof_body(net->in, -1);
    for (int t = 0; t < nnz; ++t) {
        block_of.emplace(M.mus_body[t], 0);
        dof_body[M.mus_dof[t]] = M.mus_body[t];
    }
    const int nj = (int)block_of.size(), H = net->hid;
    constexpr int kFloor = 2;
    if (nj == 0 || nj * kFloor > H) return false;
    std::vector<int> joints;
    for (auto& kv : block_of) {
        kv.second = (int)joints.size();
        joints.push_back(kv.first);
    }
    std::vector<double> outs(nj, 0.0), ndof(nj, 0.0);
    for (int d = 0; d < net->in; ++d)
        if (dof_body[d] >= 0) ndof[block_of[dof_body[d]]] += 1.0;
    for (int k = 0; k < m; ++k) {
        std::vector<int> seen;
        for (int t = M.mus_ptr[k]; t < M.mus_ptr[k + 1]; ++t) {
            const int j = block_of[M.mus_body[t]];
            outs[j] += 1.0;   // the moment arm
            if (std::find(seen.begin(), seen.end(), j) == seen.end()) {
                seen.push_back(j);
                outs[j] += 1.0;   // the length's term of this joint
            }
        }
    }
    std::vector<double> w(nj);
    double wsum = 0.0;
    for (int j = 0; j < nj; ++j) wsum += (w[j] = std::sqrt(outs[j]) * ndof[j] * ndof[j]);
    std::vector<int> units(nj);
    int total = 0;
    for (int j = 0; j < nj; ++j) total += (units[j] = std::max(kFloor, (int)std::floor(w[j] / wsum * H)));
    while (total > H) {   // take from the largest block
        const int j = (int)(std::max_element(units.begin(), units.end()) - units.begin());
        --units[j];
        --total;
    }
    while (total < H) {   // give to the block with the most weight per unit
        int jb = 0;
        for (int j = 1; j < nj; ++j)
            if (w[j] / units[j] > w[jb] / units[jb]) jb = j;
        ++units[jb];
        ++total;
    }
    std::vector<int> b0(nj + 1, 0);
    for (int j = 0; j < nj; ++j) b0[j + 1] = b0[j] + units[j];
    mask.assign(net->n_params, 0);
    for (int j = 0; j < nj; ++j)
        for (int u = b0[j]; u < b0[j + 1]; ++u) {
            for (int d = 0; d < net->in; ++d)
                if (dof_body[d] == joints[j]) mask[net->oW1 + (size_t)u * net->inp + d] = 1;
            for (int v = b0[j]; v < b0[j + 1]; ++v) mask[net->oW2 + (size_t)u * H + v] = 1;
        }
    for (int u = 0; u < H; ++u) mask[net->ob1 + u] = mask[net->ob2 + u] = 1;
    auto read_block = [&](int row, int j) {
        for (int u = b0[j]; u < b0[j + 1]; ++u) mask[net->oW3 + (size_t)row * H + u] = 1;
    };
    for (int k = 0; k < m; ++k)
        for (int t = M.mus_ptr[k]; t < M.mus_ptr[k + 1]; ++t) {
            read_block(k, block_of[M.mus_body[t]]);        // the length
            read_block(m + t, block_of[M.mus_body[t]]);    // the moment arm R_kd
        }
    for (int r = 0; r < net->out; ++r) mask[net->ob3 + r] = 1;
    return true;
}

void surr_free(Surrogate* s) {
    if (!s) return;
    if (s->net) mlp_destroy(s->net);
    cudaFree(s->mu); cudaFree(s->sd); cudaFree(s->box_c); cudaFree(s->box_s);
    cudaFree(s->X); cudaFree(s->Y); cudaFree(s->fallback); cudaFree(s->stats); cudaFree(s->step_ctr);
    cudaFree(s->out_tmp);
    cudaFree(s->colbase); cudaFree(s->head_src); cudaFree(s->W3h); cudaFree(s->b3h); cudaFree(s->scale_h);
    cudaFree(s->shift_h);
    delete s;
}

void free_all(msim_handle h) {
    surr_free(h->sur);
    h->sur = nullptr;
    for (int i = 0; i < kMaxModels; ++i)
        if (h->d_img[i]) cudaFree(h->d_img[i]);
    cudaFree(h->q); cudaFree(h->qd); cudaFree(h->act); cudaFree(h->qdd); cudaFree(h->force); cudaFree(h->eps);
    cudaFree(h->exc_stage); cudaFree(h->env_status); cudaFree(h->gflags); cudaFree(h->queue);
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->pipe_exc[b]); cudaFree(h->pipe_out[b]);
        h->pipe_exc[b] = h->pipe_out[b] = nullptr;
        for (cudaEvent_t* ev : {&h->pipe_in[b], &h->pipe_used[b], &h->pipe_snap[b], &h->pipe_done[b]})
            if (*ev) { cudaEventDestroy(*ev); *ev = nullptr; }
    }
    if (h->pipe_up) { cudaStreamDestroy(h->pipe_up); h->pipe_up = nullptr; }
    if (h->pipe_down) { cudaStreamDestroy(h->pipe_down); h->pipe_down = nullptr; }
    cudaFree(h->obs); cudaFree(h->exc_policy); cudaFree(h->inv_fmax);
    cudaFree(h->flow_x); cudaFree(h->flow_a); cudaFree(h->flow_mu); cudaFree(h->flow_v); cudaFree(h->flow_pre);
    cudaFree(h->act_ctr);
    cudaFree(h->vm); cudaFree(h->xpos_sim); cudaFree(h->xpos_ref); cudaFree(h->delta_x); cudaFree(h->disc_out);
    if (h->timers) cudaFree(h->timers);
}

// geometry-mode launch of model i over rows [0, n_rows) of q (pitch ldq) into out (pitch ldo)
cudaError_t geometry_launch(msim_handle h, int i, const float* q, int ldq, int n_rows, float* out, int ldo,
                            cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    StepArgs a = base_args(h, i);
    const int wpe = h->wpe[i] == 1 ? 1 : 2;
    int epb = h->epb[i];
    if (wpe != h->wpe[i]) epb = std::max(1, std::min(max_epb(h, i, h->pts_smem[i], wpe), 8));
    a.wpe = wpe;
    a.envs_per_block = epb;
    a.env_begin = 0;
    a.env_end = n_rows;
    a.q = const_cast<float*>(q);
    a.qd = const_cast<float*>(q);
    a.pitch_n = ldq;
    a.act = nullptr; a.eps = nullptr; a.exc = nullptr; a.qdd_out = nullptr; a.force_out = nullptr; a.vm_out = nullptr;
    a.ev.L = out;
    a.ev.nnz_pitch = ldo;
    const size_t smem = step_smem_bytes(h->models[i].hdr, epb, h->pts_smem[i], wpe);
    const int groups = (n_rows + epb - 1) / epb;
    const int per_sm = std::max(1, step_blocks_per_sm(32 * wpe * epb, smem, wpe, uses_ext(h->models[i].hdr)));
    return launch_geom(a, std::max(1, std::min(groups, h->num_sms * per_sm)), smem, s);
}

// body-position launch of model i over rows [0, n_rows) of q (pitch ldq) into xpos [row][3 nb]
cudaError_t fk_launch(msim_handle h, int i, const float* q, int ldq, int n_rows, float* xpos, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    StepArgs a = base_args(h, i);
    const int wpe = h->wpe[i] == 1 ? 1 : 2;
    int epb = h->epb[i];
    if (wpe != h->wpe[i]) epb = std::max(1, std::min(max_epb(h, i, h->pts_smem[i], wpe), 8));
    a.wpe = wpe;
    a.envs_per_block = epb;
    a.env_begin = 0;
    a.env_end = n_rows;
    a.q = const_cast<float*>(q);
    a.qd = const_cast<float*>(q);
    a.pitch_n = ldq;
    a.act = nullptr; a.eps = nullptr; a.exc = nullptr; a.qdd_out = nullptr; a.force_out = nullptr; a.vm_out = nullptr;
    a.ev.xpos = xpos;
    a.ev.xpos_pitch = 3 * h->models[i].hdr.nb;
    const size_t smem = step_smem_bytes(h->models[i].hdr, epb, h->pts_smem[i], wpe);
    const int groups = (n_rows + epb - 1) / epb;
    const int per_sm = std::max(1, step_blocks_per_sm(32 * wpe * epb, smem, wpe, uses_ext(h->models[i].hdr)));
    return launch_fk(a, std::max(1, std::min(groups, h->num_sms * per_sm)), smem, s);
}

// Column layout of the inference head (see Surrogate): muscle records in the model image's order,
// by groups of 32 (the records one warp takes in one pass); group g's C_g = 32 (1 + its largest
// crossed-DoF count) columns hold entry s of record 32 g + l at colbase[g] + 32 s + l.
void head_layout(const ModelHost& M, int m, std::vector<int>& colbase, std::vector<int>& src) {
    const MuscleRec* mus = reinterpret_cast<const MuscleRec*>(M.blob.data() + M.hdr.o_muscle);
    colbase.clear();
    src.clear();
    for (int g0 = 0; g0 < m; g0 += 32) {
        int J = 1;
        for (int r = g0; r < std::min(m, g0 + 32); ++r) J = std::max(J, 1 + (int)mus[r].nx);
        colbase.push_back((int)src.size());
        const size_t base = src.size();
        src.resize(base + 32 * (size_t)J, -1);
        for (int r = g0; r < std::min(m, g0 + 32); ++r)
            for (int e = 0; e <= mus[r].nx; ++e)
                src[base + 32 * e + (r - g0)] = e == 0 ? mus[r].orig : m + mus[r].x0 + e - 1;
    }
}

// the inference head gathered again if the network changed since (training, msim_mlp_set)
cudaError_t surr_head(Surrogate* S, cudaStream_t s) {
    const Mlp* net = S->net;
    if (S->head_version == net->version) return cudaSuccess;
    const cudaError_t e = surr_gather_head(net->Ph + net->oW3, net->P + net->ob3, S->mu, S->sd, net->hid, S->head_src,
                                           S->cols, S->W3h, S->b3h, S->scale_h, S->shift_h, s);
    if (e == cudaSuccess) S->head_version = net->version;
    return e;
}

msim_status surrogate_step(msim_handle h, const float* exc, int n_sub, cudaStream_t s) {
    Surrogate* S = h->sur;
    if (!S || !S->trained) {
        h->err = "msim_step: learned geometry selected but no surrogate has been trained";
        return MSIM_ERR_STATE;
    }
    const Mlp* net = S->net;
    for (int k = 0; k < n_sub; ++k) {
        cudaError_t e = launch_surr_input(h->q, h->pitch_n, 0, h->n_envs, S->box_c, S->box_s, S->n, S->X, net->inp,
                                          S->step_ctr, s);
        if (e == cudaSuccess) e = surr_head(S, s);
        if (e == cudaSuccess)
            e = mlp_infer_head(S->net, S->X, net->inp, h->n_envs, S->W3h, S->b3h, S->cols, S->scale_h, S->shift_h,
                               S->Y, S->cols, s);
        if (e == cudaSuccess) {
            StepArgs a = base_args(h, 0);
            a.exc = exc;
            a.n_sub = 1;
            a.surr_Y = S->Y; a.surr_ld = S->cols;
            a.surr_colbase = S->colbase;
            a.box_c = S->box_c; a.box_s = S->box_s;
            a.fallback = S->fallback; a.surr_stats = S->stats;
            a.check_frac = S->check_frac; a.tol = S->tol;
            a.surr_seed = S->seed; a.step_ctr = S->step_ctr;
            e = launch_surr_step(a, model_grid(h, 0),
                                 step_smem_bytes(h->models[0].hdr, h->epb[0], h->pts_smem[0], h->wpe[0]), s);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "msim_step (learned geometry)");
    }
    return MSIM_OK;
}

}  // namespace

extern "C" {

int32_t msim_version(void) { return 1; }

const char* msim_last_error(msim_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

msim_status msim_create(const msim_create_args* args, msim_handle* out) {
    g_create_error.clear();
    if (!args || !out) return arg_fail(nullptr, "msim_create: NULL argument");
    *out = nullptr;
    if (args->n_models < 1 || args->n_models > kMaxModels) return arg_fail(nullptr, "n_models must be 1..8");
    if (!args->models || !args->envs_per_model) return arg_fail(nullptr, "models / envs_per_model is NULL");
    if (!(args->dt > 0.f) || !std::isfinite(args->dt)) return arg_fail(nullptr, "dt must be > 0");
    if (args->geometry_mode != 0 && args->geometry_mode != 1) return arg_fail(nullptr, "geometry_mode must be 0 or 1");
    if (args->geometry_mode == 1 && args->n_models != 1) {
        g_create_error = "geometry_mode 1 (learned geometry) needs a single-model handle";
        return MSIM_ERR_UNSUPPORTED;
    }
    msim_handle h = new msim_handle_();
    h->device = args->device;
    h->geometry_mode = args->geometry_mode;
    h->seed = (uint32_t)(args->seed ^ (args->seed >> 32));
    h->n_models = args->n_models;
    h->dt = args->dt;
    int total = 0, nmax = 0, mmax = 0;
    for (int i = 0; i < args->n_models; ++i) {
        if (args->envs_per_model[i] < 0) {
            delete h;
            return arg_fail(nullptr, "envs_per_model must be >= 0");
        }
        std::string err;
        if (!build_image(args->models[i], h->models[i], err)) {
            g_create_error = "model " + std::to_string(i) + ": " + err;
            delete h;
            return MSIM_ERR_MODEL;
        }
        h->env_begin[i] = total;
        total += args->envs_per_model[i];
        nmax = std::max(nmax, args->models[i].n_dofs);
        mmax = std::max(mmax, args->models[i].n_muscles);
    }
    h->env_begin[args->n_models] = total;
    if (total < 1 || total > (1 << 24)) {
        delete h;
        return arg_fail(nullptr, "total environments must be in [1, 2^24]");
    }
    h->n_envs = total;
    h->pitch_n = pad4(nmax);
    h->pitch_m = pad4(std::max(mmax, 1));

    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) { msim_status s = cuda_fail(nullptr, e, "cudaSetDevice"); delete h; return s; }
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, h->device);
    h->num_sms = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    h->smem_optin = (size_t)v;
    e = set_step_smem_limit(h->smem_optin);
    if (e != cudaSuccess) { msim_status s = cuda_fail(nullptr, e, "smem attribute"); delete h; return s; }

    const size_t rn = (size_t)total * h->pitch_n * sizeof(float), rm = (size_t)total * h->pitch_m * sizeof(float);
#define ALLOC(ptr, bytes)                                                        \
    do {                                                                         \
        e = cudaMalloc(&(ptr), (bytes));                                         \
        if (e != cudaSuccess) {                                                  \
            msim_status s_ = cuda_fail(nullptr, e, "cudaMalloc " #ptr);          \
            free_all(h);                                                         \
            delete h;                                                            \
            return s_;                                                           \
        }                                                                        \
    } while (0)
    ALLOC(h->q, rn); ALLOC(h->qd, rn); ALLOC(h->qdd, rn);
    ALLOC(h->act, rm); ALLOC(h->force, rm); ALLOC(h->exc_stage, rm); ALLOC(h->eps, rm);
    ALLOC(h->env_status, sizeof(uint32_t) * total);
    ALLOC(h->gflags, sizeof(uint32_t));
    ALLOC(h->queue, sizeof(uint32_t));
#ifdef MSIM_PHASE_TIMERS
    ALLOC(h->timers, sizeof(unsigned long long) * 16);
    cudaMemset(h->timers, 0, sizeof(unsigned long long) * 16);
#endif
    cudaMemset(h->q, 0, rn); cudaMemset(h->qd, 0, rn); cudaMemset(h->qdd, 0, rn);
    cudaMemset(h->act, 0, rm); cudaMemset(h->force, 0, rm); cudaMemset(h->exc_stage, 0, rm); cudaMemset(h->eps, 0, rm);
    cudaMemset(h->env_status, 0, sizeof(uint32_t) * total);
    cudaMemset(h->gflags, 0, sizeof(uint32_t));

    // device images; reference lengths L0 = L(q = 0) from the device geometry code
    float *zq = nullptr, *zm = nullptr, *Lbuf = nullptr;
    ALLOC(zq, sizeof(float) * h->pitch_n * 2);
    ALLOC(zm, sizeof(float) * h->pitch_m * 3);
    Lbuf = zm + 2 * h->pitch_m;
    cudaMemset(zq, 0, sizeof(float) * h->pitch_n * 2);
    cudaMemset(zm, 0, sizeof(float) * h->pitch_m * 3);
    for (int i = 0; i < h->n_models; ++i) {
        const ModelHost& M = h->models[i];
        ALLOC(h->d_img[i], M.blob.size());
        e = cudaMemcpy(h->d_img[i], M.blob.data(), M.blob.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && M.hdr.m > 0) {
            StepArgs a;
            std::memset(&a, 0, sizeof(a));
            a.img = h->d_img[i];
            a.stage = 2;   // the smallest staged prefix: the reference lengths of any model that fits
            a.staged_bytes = staged_bytes(M.hdr, 2);
            a.env_begin = 0; a.env_end = 1;
            a.q = zq; a.qd = zq + h->pitch_n; a.act = zm; a.exc = zm + h->pitch_m;
            a.pitch_n = h->pitch_n; a.pitch_m = h->pitch_m;
            a.env_status = h->env_status; a.gflags = h->gflags;
            a.n_sub = 1; a.dt = h->dt; a.envs_per_block = 1; a.wpe = 1;
            a.ev.L = Lbuf;
            const size_t smem = step_smem_bytes(M.hdr, 1, 2, 1);
            if (smem > h->smem_optin) {
                g_create_error = "model " + std::to_string(i) + " does not fit in shared memory";
                cudaFree(zq); cudaFree(zm); free_all(h); delete h;
                return MSIM_ERR_MODEL;
            }
            e = launch_eval(a, 1, smem, 0);
            if (e == cudaSuccess) e = launch_set_l0(h->d_img[i], Lbuf, M.hdr.m, 0);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e == cudaSuccess && M.hdr.n_tendons) {
                // a compliant tendon needs a slack length L0 - l_opt of at least 0.5 l_opt
                const msim_model_desc& dm = args->models[i];
                std::vector<float> L0(M.hdr.m);
                e = cudaMemcpy(L0.data(), Lbuf, sizeof(float) * M.hdr.m, cudaMemcpyDeviceToHost);
                for (int k = 0; e == cudaSuccess && k < M.hdr.m; ++k)
                    if (dm.muscle_tendon_strain[k] > 0.f && !(L0[k] - dm.muscle_lopt[k] >= 0.5f * dm.muscle_lopt[k])) {
                        g_create_error = "model " + std::to_string(i) + ": muscle " + std::to_string(k) +
                                         ": a compliant tendon needs a slack length L0 - l_opt >= 0.5 l_opt (L0 = " +
                                         std::to_string(L0[k]) + ")";
                        cudaFree(zq); cudaFree(zm); free_all(h); delete h;
                        return MSIM_ERR_MODEL;
                    }
            }
        }
        if (e != cudaSuccess) {
            msim_status s = cuda_fail(nullptr, e, "model image upload / L0");
            cudaFree(zq); cudaFree(zm); free_all(h); delete h;
            return s;
        }
        auto_launch(h, i);
        if (h->epb[i] < 1) {
            g_create_error = "model " + std::to_string(i) + " does not fit in shared memory";
            cudaFree(zq); cudaFree(zm); free_all(h); delete h;
            return MSIM_ERR_MODEL;
        }
    }
#undef ALLOC
    cudaFree(zq);
    cudaFree(zm);
    cudaMemset(h->gflags, 0, sizeof(uint32_t));
    cudaMemset(h->env_status, 0, sizeof(uint32_t) * total);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { msim_status s = cuda_fail(nullptr, e, "create"); free_all(h); delete h; return s; }
    *out = h;
    return MSIM_OK;
}

msim_status msim_destroy(msim_handle h) {
    if (!h) return MSIM_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return MSIM_OK;
}

msim_status msim_get_dims(msim_handle h, msim_dims* out) {
    if (!h || !out) return arg_fail(h, "msim_get_dims: NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->n_envs = h->n_envs;
    out->n_models = h->n_models;
    out->pitch_n = h->pitch_n;
    out->pitch_m = h->pitch_m;
    for (int i = 0; i <= h->n_models; ++i) out->env_begin[i] = h->env_begin[i];
    for (int i = 0; i < h->n_models; ++i) {
        const ImgHeader& hd = h->models[i].hdr;
        out->n_dofs[i] = hd.n;
        out->n_muscles[i] = hd.m;
        out->n_bodies[i] = hd.nb;
        out->nnz[i] = hd.nnz;
        out->n_packed[i] = hd.n_packed;
        out->envs_per_block[i] = h->epb[i];
        out->image_bytes[i] = hd.total_bytes;
        out->workspace_bytes_per_env[i] = ws_floats(hd, h->wpe[i]) * (int)sizeof(float);
        out->points_in_smem[i] = h->pts_smem[i];
        out->warps_per_env[i] = h->wpe[i];
    }
    return MSIM_OK;
}

msim_status msim_set_launch(msim_handle h, int32_t model, int32_t envs_per_block, int32_t stage_points,
                            int32_t warps_per_env) {
    if (!h || model < 0 || model >= h->n_models) return arg_fail(h, "msim_set_launch: bad handle or model");
    if (envs_per_block < 0 || envs_per_block > kMaxEnvsPerBlock) return arg_fail(h, "envs_per_block must be 0..16");
    if (stage_points < -1 || stage_points > 2) return arg_fail(h, "stage_points must be -1, 0, 1 or 2");
    if (warps_per_env != 0 && warps_per_env != 1 && warps_per_env != 2 && warps_per_env != 4)
        return arg_fail(h, "warps_per_env must be 0, 1, 2 or 4");
    if (envs_per_block == 0 && stage_points == -1 && warps_per_env == 0) {
        auto_launch(h, model);
        return MSIM_OK;
    }
    const int pts = stage_points == -1 ? h->pts_smem[model] : stage_points;
    const int w = warps_per_env == 0 ? h->wpe[model] : warps_per_env;
    int e = envs_per_block;
    if (e == 0) e = std::min(max_epb(h, model, pts, w), 8);
    if (e < 1 || e > max_epb(h, model, pts, w) || step_smem_bytes(h->models[model].hdr, e, pts, w) > h->smem_optin)
        return arg_fail(h, "msim_set_launch: shared memory or thread limit exceeded");
    h->epb[model] = e;
    h->pts_smem[model] = pts;
    h->wpe[model] = w;
    return MSIM_OK;
}

msim_status msim_reset(msim_handle h, const float* q0, const float* qd0, const float* act0, const int32_t* env_ids,
                       int32_t n_ids, msim_stream_t stream) {
    if (!h) return arg_fail(h, "msim_reset: NULL handle");
    if (env_ids && (n_ids < 0 || n_ids > h->n_envs)) return arg_fail(h, "msim_reset: n_ids out of range");
    if (!aligned16(q0) || !aligned16(qd0) || !aligned16(act0)) return arg_fail(h, "msim_reset: unaligned pointer");
    const int rows = env_ids ? n_ids : h->n_envs;
    cudaSetDevice(h->device);
    cudaError_t e = launch_reset(h->q, h->qd, h->act, h->eps, h->env_status, h->sur ? h->sur->fallback : nullptr, q0, qd0,
                                 act0, env_ids, rows, h->pitch_n, h->pitch_m, h->n_envs, (cudaStream_t)stream);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_reset");
}

msim_status msim_step(msim_handle h, const float* excitations, int32_t n_substeps, msim_stream_t stream) {
    if (!h || !excitations) return arg_fail(h, "msim_step: NULL argument");
    if (n_substeps < 1 || n_substeps > 100000) return arg_fail(h, "msim_step: n_substeps must be 1..100000");
    if (!aligned16(excitations)) return arg_fail(h, "msim_step: excitations not 16-byte aligned");
    cudaSetDevice(h->device);
    if (h->geometry_mode == 1) return surrogate_step(h, excitations, n_substeps, (cudaStream_t)stream);
    const cudaError_t e = launch_all(h, excitations, n_substeps, (cudaStream_t)stream);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_step launch");
}

msim_status msim_step_host(msim_handle h, const float* excitations_host, int32_t n_substeps, float* q_host,
                           float* qd_host, msim_stream_t stream) {
    if (!h || !excitations_host) return arg_fail(h, "msim_step_host: NULL argument");
    cudaSetDevice(h->device);
    const size_t rm = (size_t)h->n_envs * h->pitch_m * sizeof(float);
    const size_t rn = (size_t)h->n_envs * h->pitch_n * sizeof(float);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h->exc_stage, excitations_host, rm, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "msim_step_host H2D");
    msim_status st = msim_step(h, h->exc_stage, n_substeps, stream);
    if (st != MSIM_OK) return st;
    if (q_host) e = cudaMemcpyAsync(q_host, h->q, rn, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && qd_host) e = cudaMemcpyAsync(qd_host, h->qd, rn, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_step_host D2H");
}

msim_status msim_step_host_async(msim_handle h, const float* excitations_host, int32_t n_substeps, float* q_host,
                                 float* qd_host, msim_stream_t stream) {
    if (!h || !excitations_host) return arg_fail(h, "msim_step_host_async: NULL argument");
    if (n_substeps < 1 || n_substeps > 100000) return arg_fail(h, "msim_step_host_async: n_substeps must be 1..100000");
    cudaSetDevice(h->device);
    const size_t rm = (size_t)h->n_envs * h->pitch_m * sizeof(float);
    const size_t rn = (size_t)h->n_envs * h->pitch_n * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (!h->pipe_up) {   // first call: streams, staging slots, events
        e = cudaStreamCreateWithFlags(&h->pipe_up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->pipe_down, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaMalloc(&h->pipe_exc[b], rm);
            if (e == cudaSuccess) e = cudaMalloc(&h->pipe_out[b], 2 * rn);
            for (cudaEvent_t* ev : {&h->pipe_in[b], &h->pipe_used[b], &h->pipe_snap[b], &h->pipe_done[b]})
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "msim_step_host_async set-up");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int b = h->pipe_slot;
    h->pipe_slot ^= 1;
    // up: once the step two calls back has read this slot
    e = cudaStreamWaitEvent(h->pipe_up, h->pipe_used[b], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->pipe_exc[b], excitations_host, rm, cudaMemcpyHostToDevice, h->pipe_up);
    if (e == cudaSuccess) e = cudaEventRecord(h->pipe_in[b], h->pipe_up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->pipe_in[b], 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "msim_step_host_async upload");
    const msim_status st = msim_step(h, h->pipe_exc[b], n_substeps, stream);
    if (st != MSIM_OK) return st;
    e = cudaEventRecord(h->pipe_used[b], s);
    // snapshot of the new state into the output slot (once its previous download is done), down
    float* oq = h->pipe_out[b];
    float* oqd = oq + (size_t)h->n_envs * h->pitch_n;
    if (e == cudaSuccess && (q_host || qd_host)) {
        e = cudaStreamWaitEvent(s, h->pipe_done[b], 0);
        if (e == cudaSuccess && q_host) e = cudaMemcpyAsync(oq, h->q, rn, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && qd_host) e = cudaMemcpyAsync(oqd, h->qd, rn, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(h->pipe_snap[b], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->pipe_down, h->pipe_snap[b], 0);
        if (e == cudaSuccess && q_host) e = cudaMemcpyAsync(q_host, oq, rn, cudaMemcpyDeviceToHost, h->pipe_down);
        if (e == cudaSuccess && qd_host) e = cudaMemcpyAsync(qd_host, oqd, rn, cudaMemcpyDeviceToHost, h->pipe_down);
        if (e == cudaSuccess) e = cudaEventRecord(h->pipe_done[b], h->pipe_down);
    }
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_step_host_async download");
}

msim_status msim_host_wait(msim_handle h) {
    if (!h) return arg_fail(h, "msim_host_wait: NULL handle");
    if (!h->pipe_up) return MSIM_OK;
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->pipe_up);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->pipe_down);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_host_wait");
}

msim_status msim_get_state(msim_handle h, float* q, float* qd, float* act, float* qdd, float* muscle_force,
                           uint32_t* env_status, msim_stream_t stream) {
    if (!h) return arg_fail(h, "msim_get_state: NULL handle");
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t rn = (size_t)h->n_envs * h->pitch_n * sizeof(float);
    const size_t rm = (size_t)h->n_envs * h->pitch_m * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (q) e = cudaMemcpyAsync(q, h->q, rn, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && qd) e = cudaMemcpyAsync(qd, h->qd, rn, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && qdd) e = cudaMemcpyAsync(qdd, h->qdd, rn, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && act) e = cudaMemcpyAsync(act, h->act, rm, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && muscle_force) e = cudaMemcpyAsync(muscle_force, h->force, rm, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && env_status)
        e = cudaMemcpyAsync(env_status, h->env_status, sizeof(uint32_t) * h->n_envs, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_get_state");
}

msim_status msim_tendon_strain(msim_handle h, const float* set, float* get, msim_stream_t stream) {
    if (!h) return arg_fail(h, "msim_tendon_strain: NULL handle");
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t rm = (size_t)h->n_envs * h->pitch_m * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (set) e = cudaMemcpyAsync(h->eps, set, rm, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && get) e = cudaMemcpyAsync(get, h->eps, rm, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_tendon_strain");
}

msim_status msim_get_status(msim_handle h, uint32_t* global_flags) {
    if (!h || !global_flags) return arg_fail(h, "msim_get_status: NULL argument");
    cudaSetDevice(h->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(global_flags, h->gflags, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "msim_get_status");
    if (*global_flags & (MSIM_ENV_NONFINITE | MSIM_ENV_NOT_SPD)) return MSIM_ERR_STATE;
    if (*global_flags & MSIM_FLAG_TIMEOUT) return MSIM_ERR_TIMEOUT;
    return MSIM_OK;
}

msim_status msim_clear_status(msim_handle h, msim_stream_t stream) {
    if (!h) return arg_fail(h, "msim_clear_status: NULL handle");
    cudaSetDevice(h->device);
    cudaError_t e = cudaMemsetAsync(h->env_status, 0, sizeof(uint32_t) * h->n_envs, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->gflags, 0, sizeof(uint32_t), (cudaStream_t)stream);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_clear_status");
}

msim_status msim_eval(msim_handle h, const float* q, const float* qd, const float* act, const float* exc,
                      const msim_eval_out* out, msim_stream_t stream) {
    if (!h || !q || !qd || !act || !exc || !out) return arg_fail(h, "msim_eval: NULL argument");
    int need_nnz = 0, need_packed = 0;
    for (int i = 0; i < h->n_models; ++i) {
        need_nnz = std::max(need_nnz, h->models[i].hdr.nnz);
        need_packed = std::max(need_packed, h->models[i].hdr.n_packed);
    }
    if (out->R && out->nnz_pitch < need_nnz) return arg_fail(h, "msim_eval: nnz_pitch too small");
    if ((out->M || out->A) && out->packed_pitch < need_packed) return arg_fail(h, "msim_eval: packed_pitch too small");
    cudaSetDevice(h->device);
    for (int i = 0; i < h->n_models; ++i) {
        if (h->env_begin[i + 1] == h->env_begin[i]) continue;
        StepArgs a = base_args(h, i);
        a.q = const_cast<float*>(q);
        a.qd = const_cast<float*>(qd);
        a.act = const_cast<float*>(act);
        a.exc = exc;
        a.qdd_out = nullptr;
        a.force_out = nullptr;
        a.n_sub = 1;
        a.ev.L = out->L; a.ev.lm = out->lm; a.ev.vm = out->vm; a.ev.force = out->force; a.ev.act_next = out->act_next;
        a.ev.R = out->R; a.ev.tau_m = out->tau_m; a.ev.tau_c = out->tau_c; a.ev.tau_l = out->tau_l;
        a.ev.bias = out->bias; a.ev.rhs = out->rhs; a.ev.qdd = out->qdd; a.ev.M = out->M; a.ev.A = out->A;
        a.ev.nnz_pitch = out->nnz_pitch; a.ev.packed_pitch = out->packed_pitch;
        a.eps = const_cast<float*>(out->tendon_strain);
        a.ev.eps_next = out->tendon_strain_next;
        const cudaError_t e = launch_eval(a, model_grid(h, i),
                                          step_smem_bytes(h->models[i].hdr, h->epb[i], h->pts_smem[i], h->wpe[i]),
                                          (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "msim_eval launch");
    }
    return MSIM_OK;
}

msim_status msim_get_layout(msim_handle h, int32_t model, int32_t* dof_parent, int32_t* dof_depth,
                            int32_t* packed_row, int32_t* muscle_dof_ptr, int32_t* muscle_dof) {
    if (!h || model < 0 || model >= h->n_models) return arg_fail(h, "msim_get_layout: bad handle or model");
    const ModelHost& M = h->models[model];
    auto cp = [](int32_t* dst, const std::vector<int32_t>& v) {
        if (dst && !v.empty()) std::memcpy(dst, v.data(), sizeof(int32_t) * v.size());
    };
    cp(dof_parent, M.dof_parent);
    cp(dof_depth, M.dof_depth);
    cp(packed_row, M.packed_row);
    cp(muscle_dof_ptr, M.mus_ptr);
    cp(muscle_dof, M.mus_dof);
    return MSIM_OK;
}

msim_status msim_gemm_bf16_mn(const void* A, int32_t lda, int32_t a_mn, const void* B, int32_t ldb, int32_t b_mn,
                              const float* bias, const float* addend, int32_t ld_add, void* C, int32_t ldc,
                              int32_t M, int32_t N, int32_t K, int32_t c_bf16, int32_t act, void* Z, int32_t ldz,
                              uint32_t* err, msim_stream_t stream) {
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || (a_mn != 0 && a_mn != 1) || (b_mn != 0 && b_mn != 1) ||
        lda < (a_mn ? M : K) || ldb < (b_mn ? N : K) || ldc < N || act < 0 || act > 2 || (Z && ldz < N) ||
        (addend && ld_add < N))
        return arg_fail(nullptr, "msim_gemm_bf16: bad argument");
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = M; g.N = N; g.K = K; g.C = C; g.ldc = ldc; g.c_bf16 = c_bf16 ? 1 : 0; g.bias = bias; g.act = act;
    g.Z = Z; g.ldz = ldz; g.err = err; g.a_mn = a_mn; g.b_mn = b_mn; g.addend = addend; g.ld_add = ld_add;
    const cudaError_t e = gemm_bf16_tc(A, lda, B, ldb, g, (cudaStream_t)stream);
    if (e == cudaErrorNotSupported) {
        g_create_error = "msim_gemm_bf16: tensor-map encoding unavailable";
        return MSIM_ERR_UNSUPPORTED;
    }
    if (e == cudaErrorInvalidValue) return arg_fail(nullptr, "msim_gemm_bf16: pitch or alignment not supported");
    return e == cudaSuccess ? MSIM_OK : cuda_fail(nullptr, e, "msim_gemm_bf16");
}

msim_status msim_gemm_bf16(const void* A, int32_t lda, const void* B, int32_t ldb, const float* bias, void* C,
                           int32_t ldc, int32_t M, int32_t N, int32_t K, int32_t c_bf16, int32_t act, void* Z,
                           int32_t ldz, uint32_t* err, msim_stream_t stream) {
    return msim_gemm_bf16_mn(A, lda, 0, B, ldb, 0, bias, nullptr, 0, C, ldc, M, N, K, c_bf16, act, Z, ldz, err, stream);
}

msim_status msim_mlp_create(int32_t in, int32_t hidden, int32_t out, int32_t out_act, int32_t max_batch, uint64_t seed,
                            float out_scale, msim_mlp* outp) {
    if (!outp || in < 1 || hidden < 8 || hidden % 8 || out < 1 || max_batch < 1 || (out_act != 0 && out_act != 2))
        return arg_fail(nullptr, "msim_mlp_create: bad argument");
    *outp = nullptr;
    Mlp* m = nullptr;
    cudaError_t e = mlp_create(in, hidden, out, out_act, max_batch, &m);
    if (e == cudaSuccess) e = mlp_init(m, seed, out_scale, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        mlp_destroy(m);
        return cuda_fail(nullptr, e, "msim_mlp_create");
    }
    msim_mlp h = new msim_mlp_();
    h->m = m;
    *outp = h;
    return MSIM_OK;
}

msim_status msim_mlp_destroy(msim_mlp h) {
    if (!h) return MSIM_OK;
    if (h->borrowed) return arg_fail(nullptr, "msim_mlp_destroy: network owned by a simulator handle");
    cudaDeviceSynchronize();
    mlp_destroy(h->m);
    delete h;
    return MSIM_OK;
}

msim_status msim_mlp_layout(msim_mlp h, int64_t offsets[6], int64_t* n_params, int32_t* in_pitch, int32_t* out_pitch) {
    if (!h) return arg_fail(nullptr, "msim_mlp_layout: NULL network");
    const Mlp* m = h->m;
    if (offsets) {
        offsets[0] = (int64_t)m->oW1; offsets[1] = (int64_t)m->ob1; offsets[2] = (int64_t)m->oW2;
        offsets[3] = (int64_t)m->ob2; offsets[4] = (int64_t)m->oW3; offsets[5] = (int64_t)m->ob3;
    }
    if (n_params) *n_params = (int64_t)m->n_params;
    if (in_pitch) *in_pitch = m->inp;
    if (out_pitch) *out_pitch = m->outp;
    return MSIM_OK;
}

static float* mlp_buffer(Mlp* m, int which) {
    return which == 0 ? m->P : which == 1 ? m->G : which == 2 ? m->Am : which == 3 ? m->Av : nullptr;
}

msim_status msim_mlp_get(msim_mlp h, int32_t which, float* host, int64_t n) {
    if (!h || !host || n != (int64_t)h->m->n_params || !mlp_buffer(h->m, which))
        return arg_fail(nullptr, "msim_mlp_get: bad argument");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, mlp_buffer(h->m, which), n * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(nullptr, e, "msim_mlp_get");
}

msim_status msim_mlp_set(msim_mlp h, int32_t which, const float* host, int64_t n, int32_t adam_step) {
    if (!h || !host || n != (int64_t)h->m->n_params || !mlp_buffer(h->m, which))
        return arg_fail(nullptr, "msim_mlp_set: bad argument");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(mlp_buffer(h->m, which), host, n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && which == 0) e = mlp_sync_bf16(h->m, 0);
    if (which >= 2) h->m->adam_t = adam_step;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? MSIM_OK : cuda_fail(nullptr, e, "msim_mlp_set");
}

msim_status msim_mlp_forward(msim_mlp h, const void* X, int32_t ldx, int32_t B, float* Y, int32_t ldy,
                             msim_stream_t stream) {
    if (!h || !X || !Y || B < 1 || B > h->m->max_batch || ldx < h->m->inp || ldx % 8 || ldy < h->m->out)
        return arg_fail(nullptr, "msim_mlp_forward: bad argument");
    const cudaError_t e = mlp_infer(h->m, (const __nv_bfloat16*)X, ldx, B, Y, ldy, (cudaStream_t)stream);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(nullptr, e, "msim_mlp_forward");
}

msim_status msim_mlp_backward(msim_mlp h, const void* X, int32_t ldx, const float* T, int32_t ldt, int32_t B,
                              float* loss, msim_stream_t stream) {
    if (!h || !X || !T || B < 1 || B > h->m->max_batch || ldx < h->m->inp || ldx % 8 || ldt < h->m->out)
        return arg_fail(nullptr, "msim_mlp_backward: bad argument");
    cudaError_t e = mlp_backward(h->m, (const __nv_bfloat16*)X, ldx, T, ldt, B, (cudaStream_t)stream);
    if (e == cudaSuccess && loss) {
        float sum = 0.f;
        e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaMemcpy(&sum, h->m->loss_acc, 4, cudaMemcpyDeviceToHost);
        *loss = sum / ((float)B * (float)h->m->out);
    }
    return e == cudaSuccess ? MSIM_OK : cuda_fail(nullptr, e, "msim_mlp_backward");
}

msim_status msim_mlp_adam(msim_mlp h, float lr, float beta1, float beta2, float eps, msim_stream_t stream) {
    if (!h || !(lr > 0.f)) return arg_fail(nullptr, "msim_mlp_adam: bad argument");
    const cudaError_t e = mlp_adam(h->m, lr, beta1, beta2, eps, (cudaStream_t)stream);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(nullptr, e, "msim_mlp_adam");
}


// ------------------------------------------------------------------ learned geometry
msim_status msim_geometry(msim_handle h, int32_t model, const float* q, int32_t ldq, int32_t n_rows, float* out,
                          int32_t ld_out, msim_stream_t stream) {
    if (!h || model < 0 || model >= h->n_models || !q || !out || n_rows < 0)
        return arg_fail(h, "msim_geometry: bad argument");
    const ImgHeader& hd = h->models[model].hdr;
    if (ldq < hd.n || ld_out < hd.m + hd.nnz) return arg_fail(h, "msim_geometry: pitch too small");
    cudaSetDevice(h->device);
    const cudaError_t e = geometry_launch(h, model, q, ldq, n_rows, out, ld_out, (cudaStream_t)stream);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_geometry");
}

msim_status msim_surrogate_train(msim_handle h, int64_t n_samples, int32_t epochs, int32_t batch, float lr,
                                 msim_stream_t stream) {
    if (!h) return arg_fail(h, "msim_surrogate_train: NULL handle");
    if (h->n_models != 1) {
        h->err = "msim_surrogate_train: single-model handles only";
        return MSIM_ERR_UNSUPPORTED;
    }
    if (h->models[0].hdr.free_root) {   // the training box spans joint limits; a free root has none
        h->err = "msim_surrogate_train: models with a free root are not supported";
        return MSIM_ERR_UNSUPPORTED;
    }
    if (batch < 1 || batch > 65536 || n_samples < batch || n_samples > (int64_t)1 << 30 || epochs < 1 ||
        !(lr > 0.f) || !std::isfinite(lr))
        return arg_fail(h, "msim_surrogate_train: bad argument");
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const ImgHeader& hd = h->models[0].hdr;
    const int n = hd.n, m = hd.m, nnz = hd.nnz, out = m + nnz;
    if (m < 1) return arg_fail(h, "msim_surrogate_train: model has no muscles");
    const int inp = (n + 7) & ~7, outp = (out + 7) & ~7;
    const int64_t N = n_samples;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t need = (size_t)N * ((size_t)outp * 4 + (size_t)inp * 2) + ((size_t)64 << 20);
    if (need > free_b) {
        h->err = "msim_surrogate_train: not enough device memory for the labels";
        return MSIM_ERR_OOM;
    }
    const float margin = h->sur ? h->sur->box_margin : h->box_margin;
    const float check_frac = h->sur ? h->sur->check_frac : 0.01f, tol = h->sur ? h->sur->tol : 1e-3f;
    surr_free(h->sur);
    h->sur = nullptr;
    Surrogate* S = new Surrogate();
    S->n = n; S->m = m; S->nnz = nnz; S->out = out;
    S->seed = h->seed;
    S->box_margin = margin;
    S->check_frac = check_frac;
    S->tol = tol;
    cudaError_t e = mlp_create(n, h->surr_hidden, out, 0, std::max(batch, h->n_envs), &S->net);
    if (e == cudaSuccess) e = mlp_init(S->net, (uint64_t)h->seed * 2654435761ull + 17u, 1.f, s);
    if (e == cudaSuccess && h->surr_structured) {
        std::vector<uint8_t> mask;
        if (surrogate_mask(h->models[0], S->net, m, mask)) {
            e = mlp_set_mask(S->net, mask.data(), kSurrSpreadBias ? (uint64_t)h->seed * 0x9e3779b97f4a7c15ull + 5u : 0u,
                             s);
            S->structured = 1;
        }
    }
    auto A = [&](void** p, size_t b) {
        if (e == cudaSuccess) e = cudaMalloc(p, b);
    };
    A((void**)&S->mu, outp * 4); A((void**)&S->sd, outp * 4);
    A((void**)&S->box_c, h->pitch_n * 4); A((void**)&S->box_s, h->pitch_n * 4);
    std::vector<int> colbase, head_src;
    head_layout(h->models[0], m, colbase, head_src);
    S->cols = (int)head_src.size();
    A((void**)&S->X, (size_t)h->n_envs * inp * 2); A((void**)&S->Y, (size_t)h->n_envs * S->cols * 4);
    A((void**)&S->out_tmp, (size_t)h->n_envs * S->cols * 4);
    A((void**)&S->colbase, colbase.size() * 4); A((void**)&S->head_src, head_src.size() * 4);
    A((void**)&S->W3h, (size_t)S->cols * h->surr_hidden * 2); A((void**)&S->b3h, S->cols * 4);
    A((void**)&S->scale_h, S->cols * 4); A((void**)&S->shift_h, S->cols * 4);
    if (e == cudaSuccess) e = cudaMemcpy(S->colbase, colbase.data(), colbase.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(S->head_src, head_src.data(), head_src.size() * 4, cudaMemcpyHostToDevice);
    A((void**)&S->fallback, h->n_envs); A((void**)&S->stats, 8 * 8); A((void**)&S->step_ctr, 4);
    __nv_bfloat16* Xall = nullptr;
    float *T = nullptr, *qc = nullptr;
    double* acc = nullptr;
    const int chunk = 65536;
    A((void**)&Xall, (size_t)N * inp * 2); A((void**)&T, (size_t)N * outp * 4);
    A((void**)&qc, (size_t)chunk * h->pitch_n * 4); A((void**)&acc, (size_t)outp * 16);
    if (e == cudaSuccess) {
        // training box: joint limits widened by box_margin half-ranges on each side; +-pi without limits
        std::vector<float> c(h->pitch_n, 0.f), sc(h->pitch_n, 1.f);
        const DofRec* D = reinterpret_cast<const DofRec*>(h->models[0].blob.data() + hd.o_dof);
        for (int d = 0; d < n; ++d) {
            if (D[d].lo < D[d].hi) {
                c[d] = 0.5f * (D[d].lo + D[d].hi);
                sc[d] = 0.5f * (D[d].hi - D[d].lo) * (1.f + margin);
            } else {
                c[d] = 0.f;
                sc[d] = 3.14159265f;
            }
        }
        e = cudaMemcpyAsync(S->box_c, c.data(), h->pitch_n * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(S->box_s, sc.data(), h->pitch_n * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors go out of scope
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(S->fallback, 0, h->n_envs, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->stats, 0, 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->step_ctr, 0, 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, (size_t)outp * 16, s);
    // labels from the exact geometry kernel, chunk by chunk
    for (int64_t r0 = 0; r0 < N && e == cudaSuccess; r0 += chunk) {
        const int rows = (int)std::min<int64_t>(chunk, N - r0);
        e = surr_sample(qc, h->pitch_n, Xall + (size_t)r0 * inp, inp, rows, n, S->box_c, S->box_s, S->seed,
                        (uint64_t)r0, s);
        if (e == cudaSuccess) e = geometry_launch(h, 0, qc, h->pitch_n, rows, T + (size_t)r0 * outp, outp, s);
        if (e == cudaSuccess) e = surr_col_stats(T + (size_t)r0 * outp, outp, rows, out, acc, s);
    }
    if (e == cudaSuccess) e = surr_finalize(acc, out, outp, (double)N, kSurrSdFloor, S->mu, S->sd, s);
    if (e == cudaSuccess) e = surr_normalize(T, outp, N, out, S->mu, S->sd, s);
    // minibatches: contiguous blocks of the i.i.d. samples, visited in an affine-permuted order
    // per epoch; cosine learning-rate decay from lr to lr / 100
    const int64_t nb = N / batch;
    const int64_t total_it = nb * epochs;
    int64_t it = 0;
    float last = 0.f;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        uint32_t ctr[4] = {(uint32_t)ep, 0x7e57u, 0u, 0u};
        philox4x32_10(ctr, S->seed, 0x51ed270bu);
        int64_t mult = 1 + 2 * (int64_t)(ctr[0] % 1024);
        while (std::gcd(mult, nb) != 1) mult += 2;
        const int64_t off = (int64_t)(ctr[1] % (uint32_t)nb);
        for (int64_t k = 0; k < nb && e == cudaSuccess; ++k, ++it) {
            const int64_t b = (mult * k + off) % nb;
            const double frac = (double)it / (double)std::max<int64_t>(total_it - 1, 1);
            const float lr_t = (float)(lr * (0.01 + 0.99 * 0.5 * (1.0 + std::cos(3.14159265358979 * frac))));
            e = mlp_backward(S->net, Xall + (size_t)b * batch * inp, inp, T + (size_t)b * batch * outp, outp, batch, s);
            if (e == cudaSuccess) e = mlp_adam(S->net, lr_t, 0.9f, 0.999f, 1e-8f, s);
        }
        if (e == cudaSuccess && ep == epochs - 1) {
            float sum = 0.f;
            e = cudaStreamSynchronize(s);
            if (e == cudaSuccess) e = cudaMemcpy(&sum, S->net->loss_acc, 4, cudaMemcpyDeviceToHost);
            last = sum / ((float)batch * (float)out);
        }
    }
    uint32_t gemm_err = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&gemm_err, S->net->err, 4, cudaMemcpyDeviceToHost);
    cudaFree(Xall); cudaFree(T); cudaFree(qc); cudaFree(acc);
    if (e != cudaSuccess || gemm_err) {
        const msim_status st = e != cudaSuccess ? cuda_fail(h, e, "msim_surrogate_train") : MSIM_ERR_TIMEOUT;
        if (gemm_err) h->err = "msim_surrogate_train: a GEMM wait ran out";
        surr_free(S);
        return st;
    }
    S->loss = last;
    S->trained = 1;
    h->sur = S;
    h->sur_view.m = S->net;
    h->sur_view.borrowed = true;
    return MSIM_OK;
}

msim_status msim_set_geometry_mode(msim_handle h, int32_t mode) {
    if (!h || (mode != 0 && mode != 1)) return arg_fail(h, "msim_set_geometry_mode: mode must be 0 or 1");
    if (mode == 1 && h->n_models != 1) {
        h->err = "msim_set_geometry_mode: learned geometry needs a single-model handle";
        return MSIM_ERR_UNSUPPORTED;
    }
    if (mode == 1 && (!h->sur || !h->sur->trained)) {
        h->err = "msim_set_geometry_mode: no trained surrogate (msim_surrogate_train)";
        return MSIM_ERR_STATE;
    }
    h->geometry_mode = mode;
    return MSIM_OK;
}

msim_status msim_surrogate_set_box(msim_handle h, float margin) {
    if (!h || !(margin >= 0.f && margin <= 10.f)) return arg_fail(h, "msim_surrogate_set_box: margin in [0, 10]");
    h->box_margin = margin;
    if (h->sur) h->sur->box_margin = margin;   // takes effect at the next msim_surrogate_train
    return MSIM_OK;
}

msim_status msim_surrogate_set_width(msim_handle h, int32_t hidden) {
    if (!h || hidden < 64 || hidden > 4096 || hidden % 64)
        return arg_fail(h, "msim_surrogate_set_width: hidden must be a multiple of 64 in [64, 4096]");
    h->surr_hidden = hidden;   // takes effect at the next msim_surrogate_train
    return MSIM_OK;
}

msim_status msim_surrogate_set_structure(msim_handle h, int32_t structured) {
    if (!h || (structured != 0 && structured != 1))
        return arg_fail(h, "msim_surrogate_set_structure: structured must be 0 or 1");
    h->surr_structured = structured;   // takes effect at the next msim_surrogate_train
    return MSIM_OK;
}

msim_status msim_surrogate_set_check(msim_handle h, float check_frac, float tol) {
    if (!h || !(check_frac >= 0.f && check_frac <= 1.f) || !(tol > 0.f) || !std::isfinite(tol))
        return arg_fail(h, "msim_surrogate_set_check: check_frac in [0, 1], tol > 0");
    if (!h->sur) {
        h->err = "msim_surrogate_set_check: no trained surrogate";
        return MSIM_ERR_STATE;
    }
    h->sur->check_frac = check_frac;
    h->sur->tol = tol;
    return MSIM_OK;
}

msim_status msim_surrogate_stats(msim_handle h, msim_surrogate_info* out, int32_t reset_counters) {
    if (!h || !out) return arg_fail(h, "msim_surrogate_stats: NULL argument");
    std::memset(out, 0, sizeof(*out));
    if (!h->sur) return MSIM_OK;
    cudaSetDevice(h->device);
    unsigned long long c[8] = {};
    std::vector<uint8_t> fb(h->n_envs);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c, h->sur->stats, sizeof(c), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(fb.data(), h->sur->fallback, h->n_envs, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset_counters) e = cudaMemset(h->sur->stats, 0, sizeof(c));
    if (e != cudaSuccess) return cuda_fail(h, e, "msim_surrogate_stats");
    out->env_substeps = c[0]; out->learned = c[1]; out->out_of_box = c[2];
    out->flagged = c[3]; out->checked = c[4]; out->check_failed = c[5];
    uint32_t bits = (uint32_t)c[6];
    std::memcpy(&out->max_check_error, &bits, 4);
    out->train_loss = h->sur->loss;
    int nf = 0;
    for (uint8_t v : fb) nf += v != 0;
    out->flagged_envs = nf;
    out->trained = h->sur->trained;
    out->structured = h->sur->structured;
    out->hidden = h->sur->net ? h->sur->net->hid : 0;
    return MSIM_OK;
}

msim_status msim_surrogate_network(msim_handle h, msim_mlp* net) {
    if (!h || !net) return arg_fail(h, "msim_surrogate_network: NULL argument");
    *net = nullptr;
    if (!h->sur || !h->sur->trained) {
        h->err = "msim_surrogate_network: no trained surrogate";
        return MSIM_ERR_STATE;
    }
    *net = &h->sur_view;
    return MSIM_OK;
}

msim_status msim_surrogate_predict(msim_handle h, const float* q, int32_t ldq, int32_t n_rows, float* out,
                                   int32_t ld_out, msim_stream_t stream) {
    if (!h || !q || !out || n_rows < 0) return arg_fail(h, "msim_surrogate_predict: bad argument");
    Surrogate* S = h->sur;
    if (!S || !S->trained) {
        h->err = "msim_surrogate_predict: no trained surrogate";
        return MSIM_ERR_STATE;
    }
    if (ldq < S->n || ld_out < S->out) return arg_fail(h, "msim_surrogate_predict: pitch too small");
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    for (int r0 = 0; r0 < n_rows && e == cudaSuccess; r0 += h->n_envs) {
        const int rows = std::min(h->n_envs, n_rows - r0);
        e = launch_surr_input(q, ldq, r0, rows, S->box_c, S->box_s, S->n, S->X, S->net->inp, nullptr, s);
        if (e == cudaSuccess) e = surr_head(S, s);
        if (e == cudaSuccess)
            e = mlp_infer_head(S->net, S->X, S->net->inp, rows, S->W3h, S->b3h, S->cols, S->scale_h, S->shift_h,
                               S->out_tmp, S->cols, s);
        if (e == cudaSuccess)
            e = surr_unpermute(S->out_tmp, S->cols, rows, S->head_src, S->cols, out + (size_t)r0 * ld_out, ld_out, s);
    }
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_surrogate_predict");
}

// ------------------------------------------------------------------ policy in the loop
msim_status msim_policy_attach(msim_handle h, msim_mlp policy) {
    if (!h) return arg_fail(h, "msim_policy_attach: NULL handle");
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->obs); cudaFree(h->exc_policy); cudaFree(h->inv_fmax);
    h->obs = nullptr; h->exc_policy = nullptr; h->inv_fmax = nullptr; h->policy = nullptr;
    msim_flow_attach(h, nullptr, 0, 0.f, 0.f);   // a flow network is bound to its sampler
    if (!policy) return MSIM_OK;   // detach
    if (h->n_models != 1) {
        h->err = "msim_policy_attach: single-model handles only";
        return MSIM_ERR_UNSUPPORTED;
    }
    const ImgHeader& hd = h->models[0].hdr;
    Mlp* p = policy->m;
    if (p->in < 2 * hd.n + 2 * hd.m || p->out != hd.m || p->max_batch < h->n_envs)
        return arg_fail(h, "msim_policy_attach: policy needs in >= 2 n + 2 m, out = m, max_batch >= n_envs");
    std::vector<float> inv(h->pitch_m, 0.f);
    const MuscleRec* M = reinterpret_cast<const MuscleRec*>(h->models[0].blob.data() + hd.o_muscle);
    for (int r = 0; r < hd.m; ++r) inv[M[r].orig] = 1.f / M[r].fmax;
    cudaError_t e = cudaMalloc(&h->obs, (size_t)h->n_envs * p->inp * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&h->exc_policy, (size_t)h->n_envs * h->pitch_m * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->inv_fmax, (size_t)h->pitch_m * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(h->inv_fmax, inv.data(), inv.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->exc_policy, 0, (size_t)h->n_envs * h->pitch_m * sizeof(float));
    if (e != cudaSuccess) {
        cudaFree(h->obs); cudaFree(h->exc_policy); cudaFree(h->inv_fmax);
        h->obs = nullptr; h->exc_policy = nullptr; h->inv_fmax = nullptr;
        return cuda_fail(h, e, "msim_policy_attach");
    }
    h->policy = p;
    return MSIM_OK;
}

msim_status msim_policy_step(msim_handle h, int32_t n_substeps_per_act, int32_t n_acts, msim_stream_t stream) {
    if (!h) return arg_fail(h, "msim_policy_step: NULL handle");
    if (!h->policy) {
        h->err = "msim_policy_step: no policy attached (msim_policy_attach)";
        return MSIM_ERR_STATE;
    }
    if (n_substeps_per_act < 1 || n_substeps_per_act > 100000 || n_acts < 0)
        return arg_fail(h, "msim_policy_step: n_substeps_per_act 1..100000, n_acts >= 0");
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const ImgHeader& hd = h->models[0].hdr;
    Mlp* p = h->policy;
    Mlp* f = h->flow;
    const int E = h->n_envs, m = hd.m;
    for (int k = 0; k < n_acts; ++k) {
        cudaError_t e = launch_obs(h->q, h->qd, h->act, h->force, h->inv_fmax, h->pitch_n, h->pitch_m, hd.n, hd.m,
                                   h->n_envs, h->obs, p->inp, s);
        if (!f) {
            if (e == cudaSuccess) e = mlp_infer(p, h->obs, p->inp, E, h->exc_policy, h->pitch_m, s);
        } else {
            // a0 = mu(s) + sigma eps; a += dt psi(t, s, a) for N steps; u = clamp(a, 0, 1)
            const int off = p->in;   // the flow input holds the observation columns first
            if (e == cudaSuccess) e = mlp_infer(p, h->obs, p->inp, E, h->flow_mu, h->pitch_m, s);
            if (e == cudaSuccess)
                e = launch_flow_init(h->flow_mu, h->pitch_m, h->flow_a, h->pitch_m, E, m, h->flow_sigma, h->seed,
                                     h->act_ctr, s);
            if (e == cudaSuccess) e = launch_copy_cols(h->obs, p->inp, E, p->in, h->flow_x, f->inp, s);
            // the observation columns of the flow input do not change over the Euler steps: their
            // share of the first layer is formed at the first step and reused
            // (each Euler step's update also writes the next step's [a | t] input columns)
            if (e == cudaSuccess && h->flow_steps > 0)
                e = launch_flow_input(h->flow_a, h->pitch_m, E, m, 0.f, h->flow_x, f->inp, off, s);
            for (int j = 0; j < h->flow_steps && e == cudaSuccess; ++j) {
                e = h->flow_split ? mlp_infer_split(f, h->flow_x, f->inp, E, h->flow_split, h->flow_pre, j == 0,
                                                    h->flow_v, f->outp, s)
                                  : mlp_infer(f, h->flow_x, f->inp, E, h->flow_v, f->outp, s);
                if (e == cudaSuccess)
                    e = launch_flow_axpy(h->flow_a, h->pitch_m, h->flow_v, f->outp, E, m, h->flow_dt,
                                         j + 1 == h->flow_steps ? h->exc_policy : nullptr, h->pitch_m,
                                         j + 1 == h->flow_steps ? nullptr : h->flow_x, f->inp, off,
                                         (float)(j + 1) * h->flow_dt, s);
            }
            if (e == cudaSuccess && h->flow_steps == 0)   // no refinement: u = clamp(a0)
                e = launch_flow_axpy(h->flow_a, h->pitch_m, h->flow_v, f->outp, E, m, 0.f, h->exc_policy, h->pitch_m,
                                     nullptr, 0, 0, 0.f, s);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "msim_policy_step (policy)");
        const msim_status st = msim_step(h, h->exc_policy, n_substeps_per_act, stream);
        if (st != MSIM_OK) return st;
    }
    return MSIM_OK;
}

msim_status msim_policy_excitations(msim_handle h, float* out, msim_stream_t stream) {
    if (!h || !out) return arg_fail(h, "msim_policy_excitations: NULL argument");
    if (!h->exc_policy) {
        h->err = "msim_policy_excitations: no policy attached";
        return MSIM_ERR_STATE;
    }
    cudaSetDevice(h->device);
    const cudaError_t e = cudaMemcpyAsync(out, h->exc_policy, (size_t)h->n_envs * h->pitch_m * sizeof(float),
                                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_policy_excitations");
}

msim_status msim_flow_attach(msim_handle h, msim_mlp flow, int32_t n_steps, float dt, float sigma) {
    if (!h) return arg_fail(h, "msim_flow_attach: NULL handle");
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->flow_x); cudaFree(h->flow_a); cudaFree(h->flow_mu); cudaFree(h->flow_v); cudaFree(h->act_ctr);
    cudaFree(h->flow_pre);
    h->flow_x = nullptr; h->flow_a = nullptr; h->flow_mu = nullptr; h->flow_v = nullptr; h->act_ctr = nullptr;
    h->flow_pre = nullptr;
    h->flow_split = 0;
    h->flow = nullptr;
    if (!flow) return MSIM_OK;   // detach
    if (!h->policy) {
        h->err = "msim_flow_attach: attach the initial sampler first (msim_policy_attach)";
        return MSIM_ERR_STATE;
    }
    const ImgHeader& hd = h->models[0].hdr;
    Mlp* f = flow->m;
    const int m = hd.m;
    if (f->in != h->policy->in + m + 1 || f->out != m || f->max_batch < h->n_envs || h->policy->out != m)
        return arg_fail(h, "msim_flow_attach: flow needs in = policy in + m + 1, out = m, max_batch >= n_envs");
    if (n_steps < 0 || n_steps > 1000 || !(dt >= 0.f) || !(sigma >= 0.f) || !std::isfinite(dt) || !std::isfinite(sigma))
        return arg_fail(h, "msim_flow_attach: 0 <= n_steps <= 1000, dt >= 0, sigma >= 0");
    cudaError_t e = cudaMalloc(&h->flow_x, (size_t)h->n_envs * f->inp * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&h->flow_a, (size_t)h->n_envs * h->pitch_m * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->flow_mu, (size_t)h->n_envs * h->pitch_m * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->flow_v, (size_t)h->n_envs * f->outp * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->act_ctr, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(h->flow_x, 0, (size_t)h->n_envs * f->inp * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMemset(h->flow_a, 0, (size_t)h->n_envs * h->pitch_m * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(h->flow_mu, 0, (size_t)h->n_envs * h->pitch_m * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(h->flow_v, 0, (size_t)h->n_envs * f->outp * sizeof(float));
    // first-layer columns shared by every Euler step: the observation's, rounded down to 8
    const int split = (h->policy->in / 8) * 8;
    if (e == cudaSuccess && split >= 8 && split < f->in) {
        e = cudaMalloc(&h->flow_pre, (size_t)h->n_envs * f->hid * sizeof(float));
        if (e == cudaSuccess) h->flow_split = split;
    }
    if (e == cudaSuccess) e = cudaMemset(h->act_ctr, 0, sizeof(uint32_t));
    if (e != cudaSuccess) {
        cudaFree(h->flow_x); cudaFree(h->flow_a); cudaFree(h->flow_mu); cudaFree(h->flow_v); cudaFree(h->act_ctr);
        cudaFree(h->flow_pre);
        h->flow_x = nullptr; h->flow_a = nullptr; h->flow_mu = nullptr; h->flow_v = nullptr; h->act_ctr = nullptr;
        h->flow_pre = nullptr;
        h->flow_split = 0;
        return cuda_fail(h, e, "msim_flow_attach");
    }
    h->flow = f;
    h->flow_steps = n_steps;
    h->flow_dt = dt;
    h->flow_sigma = sigma;
    return MSIM_OK;
}

msim_status msim_flow_actions(msim_handle h, float* a0, float* a, msim_stream_t stream) {
    if (!h || (!a0 && !a)) return arg_fail(h, "msim_flow_actions: NULL argument");
    if (!h->flow) {
        h->err = "msim_flow_actions: no flow attached";
        return MSIM_ERR_STATE;
    }
    cudaSetDevice(h->device);
    const size_t bytes = (size_t)h->n_envs * h->pitch_m * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (a0) e = cudaMemcpyAsync(a0, h->flow_mu, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (e == cudaSuccess && a) e = cudaMemcpyAsync(a, h->flow_a, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_flow_actions");
}

// ------------------------------------------------------------------ imitation reward
msim_status msim_reward_attach(msim_handle h, msim_mlp disc, float w_power) {
    if (!h) return arg_fail(h, "msim_reward_attach: NULL handle");
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->vm); cudaFree(h->xpos_sim); cudaFree(h->xpos_ref); cudaFree(h->delta_x); cudaFree(h->disc_out);
    h->vm = nullptr; h->xpos_sim = nullptr; h->xpos_ref = nullptr; h->delta_x = nullptr; h->disc_out = nullptr;
    h->disc = nullptr;
    if (!disc) return MSIM_OK;   // detach (the step stops writing fibre velocities)
    if (h->n_models != 1) {
        h->err = "msim_reward_attach: single-model handles only";
        return MSIM_ERR_UNSUPPORTED;
    }
    const ImgHeader& hd = h->models[0].hdr;
    Mlp* d = disc->m;
    if (d->in != hd.n + 3 * hd.nb || d->out != 1 || d->out_act != 2 || d->max_batch < h->n_envs)
        return arg_fail(h, "msim_reward_attach: discriminator needs in = n + 3 nb, out = 1 (sigmoid), "
                           "max_batch >= n_envs");
    if (!std::isfinite(w_power)) return arg_fail(h, "msim_reward_attach: w_power must be finite");
    const size_t E = (size_t)h->n_envs;
    cudaError_t e = cudaMalloc(&h->vm, E * h->pitch_m * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->xpos_sim, E * 3 * hd.nb * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->xpos_ref, E * 3 * hd.nb * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->delta_x, E * d->inp * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&h->disc_out, E * d->outp * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(h->vm, 0, E * h->pitch_m * sizeof(float));
    if (e != cudaSuccess) {
        cudaFree(h->vm); cudaFree(h->xpos_sim); cudaFree(h->xpos_ref); cudaFree(h->delta_x); cudaFree(h->disc_out);
        h->vm = nullptr; h->xpos_sim = nullptr; h->xpos_ref = nullptr; h->delta_x = nullptr; h->disc_out = nullptr;
        return cuda_fail(h, e, "msim_reward_attach");
    }
    h->disc = d;
    h->w_power = w_power;
    return MSIM_OK;
}

msim_status msim_reward(msim_handle h, const float* q_ref, float* reward, float* parts, float* delta, int32_t ld_delta,
                        msim_stream_t stream) {
    if (!h || !q_ref || !reward) return arg_fail(h, "msim_reward: NULL argument");
    if (!h->disc) {
        h->err = "msim_reward: no discriminator attached (msim_reward_attach)";
        return MSIM_ERR_STATE;
    }
    const ImgHeader& hd = h->models[0].hdr;
    if (delta && ld_delta < hd.n + 3 * hd.nb) return arg_fail(h, "msim_reward: ld_delta < n + 3 nb");
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    Mlp* d = h->disc;
    const int E = h->n_envs;
    cudaError_t e = fk_launch(h, 0, h->q, h->pitch_n, E, h->xpos_sim, s);
    if (e == cudaSuccess) e = fk_launch(h, 0, q_ref, h->pitch_n, E, h->xpos_ref, s);
    if (e == cudaSuccess)
        e = launch_delta(h->q, q_ref, h->pitch_n, h->xpos_sim, h->xpos_ref, hd.n, hd.nb, E, h->delta_x, d->inp, delta,
                         ld_delta, s);
    if (e == cudaSuccess) e = mlp_infer(d, h->delta_x, d->inp, E, h->disc_out, d->outp, s);
    if (e == cudaSuccess)
        e = launch_reward(h->disc_out, d->outp, h->force, h->vm, h->pitch_m, hd.m, E, h->w_power, reward, parts, s);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_reward");
}

msim_status msim_body_positions(msim_handle h, const float* q, int32_t ldq, int32_t n_rows, float* xpos,
                                msim_stream_t stream) {
    if (!h || !q || !xpos || n_rows < 0) return arg_fail(h, "msim_body_positions: bad argument");
    if (h->n_models != 1) {
        h->err = "msim_body_positions: single-model handles only";
        return MSIM_ERR_UNSUPPORTED;
    }
    if (ldq < h->models[0].hdr.n) return arg_fail(h, "msim_body_positions: ldq < n");
    cudaSetDevice(h->device);
    const cudaError_t e = fk_launch(h, 0, q, ldq, n_rows, xpos, (cudaStream_t)stream);
    return e == cudaSuccess ? MSIM_OK : cuda_fail(h, e, "msim_body_positions");
}

#ifdef MSIM_PHASE_TIMERS
// Profiling builds only: per-phase cycle sums over all warps since the last reset.
MSIM_API msim_status msim_debug_phase_cycles(msim_handle h, unsigned long long* out8, int32_t reset) {
    if (!h || !out8 || !h->timers) return arg_fail(h, "msim_debug_phase_cycles: unavailable");
    cudaDeviceSynchronize();
    cudaMemcpy(out8, h->timers, sizeof(unsigned long long) * 16, cudaMemcpyDeviceToHost);
    if (reset) cudaMemset(h->timers, 0, sizeof(unsigned long long) * 16);
    return MSIM_OK;
}
#endif

}  // extern "C"
