// sl1m_refine.cpp -- adaptive quadtree refinement of the pixel set
// (Hardy 2013, Sect. 4.4: solve on a coarse grid first, then split the
// pixels that hold emission and solve again, repeatedly; in the paper's
// example every pixel above 1% of the maximum is split, level by level, from
// 64" to 2").
//
// Each level is an ordinary solve on the GPU (power iteration for L, FISTA);
// between levels the host splits every pixel above refine_frac * peak into
// its four quadrant children at half the spacing and starts the next solve
// from the parent's flux shared equally among its children.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sl1m_host.h"

extern "C" int sl1m_solve_refine(sl1m_problem* prob, const sl1m_solve_opts* o, const sl1m_refine_opts* ro,
                                 double delta0, sl1m_refine_stats* rs)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    if (!o || !ro || !(delta0 > 0) || ro->levels < 0 || ro->levels > 16 || !(ro->refine_frac > 0) ||
        !(ro->refine_frac < 1))
        return sl1m_fail(ctx, SL1M_ERR_ARG, "bad refinement options");
    if (prob->n_pix <= 0 || prob->n_vis <= 0) return sl1m_fail(ctx, SL1M_ERR_STATE, "problem incomplete");
    if (!prob->kind.empty())
        for (int k : prob->kind)
            if (k != 0) return sl1m_fail(ctx, SL1M_ERR_ARG, "refinement works on Dirac pixels");
    if (prob->n_ant > 0) return sl1m_fail(ctx, SL1M_ERR_ARG, "refinement of problems with gains is not supported");
    std::vector<double> lm = prob->lm;
    std::vector<double> delta(prob->n_pix, delta0);
    std::vector<double> img(prob->n_pix), x0;
    sl1m_solve_opts oo = *o;
    if (rs) {
        rs->levels_done = 0;
        rs->total_pair_evals = 0.0;
    }
    for (int level = 0; level <= ro->levels; ++level) {
        oo.x0 = level == 0 ? o->x0 : x0.data();
        sl1m_solve_stats st;
        img.assign(prob->n_pix, 0.0);
        int rc = sl1m_solve(prob, &oo, img.data(), &st);
        if (rc != SL1M_OK) return rc;
        if (rs) {
            rs->levels_done = level + 1;
            rs->n_pix[level] = prob->n_pix;
            rs->iters[level] = st.iters;
            rs->power_iters[level] = st.power_iters;
            rs->total_pair_evals += (2.0 * st.iters + 2.0 * st.power_iters + 2.0) * (double)prob->n_vis *
                                    (double)prob->n_pix;
            rs->last = st;
        }
        if (level == ro->levels) break;
        const double peak = *std::max_element(img.begin(), img.end());
        if (!(peak > 0)) break;
        const double thr = ro->refine_frac * peak;
        std::vector<double> nlm, nd;
        x0.clear();
        bool any = false;
        for (int64_t j = 0; j < prob->n_pix; ++j) {
            const double l = lm[2 * j], m = lm[2 * j + 1], d = delta[j];
            if (img[j] > thr) {
                any = true;
                const double q = 0.25 * d;
                const double off[4][2] = {{-q, -q}, {q, -q}, {-q, q}, {q, q}};
                for (auto& of : off) {
                    const double cl = l + of[0], cm = m + of[1];
                    if (!(cl * cl + cm * cm < 1.0)) continue;
                    nlm.push_back(cl);
                    nlm.push_back(cm);
                    nd.push_back(0.5 * d);
                    x0.push_back(0.25 * img[j]);
                }
            } else if (ro->keep_unrefined) {
                nlm.push_back(l);
                nlm.push_back(m);
                nd.push_back(d);
                x0.push_back(img[j]);
            }
        }
        if (!any) break;
        const int64_t n_new = (int64_t)nd.size();
        int rc2 = sl1m_set_pixels(prob, n_new, nlm.data(), nullptr, nullptr);
        if (rc2 != SL1M_OK) return rc2;
        lm.swap(nlm);
        delta.swap(nd);
    }
    prob->last_img = img;
    if (rs) rs->final_n_pix = prob->n_pix;
    return SL1M_OK;
}

extern "C" int sl1m_get_solution(const sl1m_problem* prob, int64_t* n_pix, double* lm_out, double* img_out)
{
    if (!prob) return SL1M_ERR_ARG;
    if (n_pix) *n_pix = prob->n_pix;
    if (lm_out) std::copy(prob->lm.begin(), prob->lm.end(), lm_out);
    if (img_out) {
        if ((int64_t)prob->last_img.size() != prob->n_pix)
            return sl1m_fail(prob->ctx, SL1M_ERR_STATE, "no refined solution for the current pixels");
        std::copy(prob->last_img.begin(), prob->last_img.end(), img_out);
    }
    return SL1M_OK;
}
