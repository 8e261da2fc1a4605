// Execution-plan generation on the host (Section 4.2) and its flattening into
// the sequential execution path evaluated on the GPU (Section 5.1).
//
//   order      : predicates by cost-effectiveness (1 - sp) / cost, descending,
//                ties to the lower predicate id ("Ordering scheme");
//   tree       : every MD's predicates, in that order, inserted from the root,
//                reusing a child edge with the same predicate ("Constructing an
//                execution tree");
//   wp(phi)    : product of sp over the MD's predicates (independence);
//   score(e)   : max wp over the MDs whose path contains e ("Edge score");
//   DFS        : children in decreasing score, ties to the child created first;
//   program    : the DFS edge sequence, each predicate kept at its first
//                occurrence (its result is reused afterwards, "Reusing
//                computation"), minus the predicates decided by blocking; an
//                MD's checkpoint sits at its last remaining predicate.
#include <stdint.h>

#include <algorithm>
#include <functional>
#include <memory>
#include <vector>

#include "hb_internal.h"

namespace hb {

struct PlanNode {
    int pred = -1;
    int first_md = -1;
    double score = 0.0;
    std::vector<int> mds;
    std::vector<int> leaf_mds;
    std::vector<std::unique_ptr<PlanNode>> kids;
};

PlanResult make_plan(int n_preds, const double *sp, const double *cost, const std::vector<std::vector<int>> &mds,
                     const std::vector<uint8_t> &skip) {
    PlanResult R;
    std::vector<double> ce(n_preds);
    for (int p = 0; p < n_preds; p++) ce[p] = (1.0 - sp[p]) / cost[p];
    auto better = [&](int a, int b) {
        if (ce[a] != ce[b]) return ce[a] > ce[b];
        return a < b;
    };
    R.pred_order.resize(n_preds);
    for (int p = 0; p < n_preds; p++) R.pred_order[p] = p;
    std::stable_sort(R.pred_order.begin(), R.pred_order.end(), better);

    PlanNode root;
    for (int m = 0; m < (int)mds.size(); m++) {
        std::vector<int> seq;
        for (int p : mds[m])
            if (std::find(seq.begin(), seq.end(), p) == seq.end()) seq.push_back(p);
        std::stable_sort(seq.begin(), seq.end(), better);
        PlanNode *node = &root;
        for (int p : seq) {
            PlanNode *child = nullptr;
            for (auto &k : node->kids)
                if (k->pred == p) {
                    child = k.get();
                    break;
                }
            if (!child) {
                node->kids.emplace_back(new PlanNode());
                child = node->kids.back().get();
                child->pred = p;
                child->first_md = m;
            }
            child->mds.push_back(m);
            node = child;
        }
        node->leaf_mds.push_back(m);
    }
    R.wp.resize(mds.size());
    for (size_t m = 0; m < mds.size(); m++) {
        double w = 1.0;
        for (int p : mds[m]) w *= sp[p];
        R.wp[m] = w;
    }
    std::function<void(PlanNode *)> score = [&](PlanNode *n) {
        for (auto &k : n->kids) {
            double s = 0.0;
            bool first = true;
            for (int m : k->mds) {
                if (first || R.wp[m] > s) s = R.wp[m];
                first = false;
            }
            k->score = s;
            score(k.get());
        }
    };
    score(&root);
    std::vector<int> path;   // >= 0: predicate; < 0: checkpoint of MD -(v+1)
    std::function<void(PlanNode *)> dfs = [&](PlanNode *n) {
        for (int m : n->leaf_mds) path.push_back(-(m + 1));
        std::vector<PlanNode *> order;
        for (auto &k : n->kids) order.push_back(k.get());
        std::stable_sort(order.begin(), order.end(), [](PlanNode *a, PlanNode *b) {
            if (a->score != b->score) return a->score > b->score;
            return a->first_md < b->first_md;
        });
        for (PlanNode *k : order) {
            path.push_back(k->pred);
            dfs(k);
        }
    };
    dfs(&root);
    std::vector<int> pos(n_preds, -1);
    for (int v : path) {
        if (v < 0) {
            R.md_order.push_back(-v - 1);
        } else if (pos[v] < 0 && !(v < (int)skip.size() && skip[v])) {
            pos[v] = (int)R.program.size();
            R.program.push_back(v);
        }
    }
    R.cp.assign(mds.size(), -1);
    for (size_t m = 0; m < mds.size(); m++)
        for (int p : mds[m])
            if (pos[p] > R.cp[m]) R.cp[m] = pos[p];
    return R;
}

}  // namespace hb

extern "C" hb_status hb_plan_order(int32_t n_preds, const double *sp, const double *cost, int32_t n_mds,
                                   const int32_t *md_start, const int32_t *md_pred, const uint8_t *skip,
                                   int32_t *program_out, int32_t *n_prog_out, int32_t *cp_out,
                                   int32_t *md_order_out) {
    if (n_preds < 0 || n_preds > HB_MAX_PREDS || n_mds < 0 || n_mds > HB_MAX_MDS || (!sp && n_preds) ||
        (!cost && n_preds) || !md_start || (!md_pred && n_mds))
        return HB_ERR_ARG;
    for (int p = 0; p < n_preds; p++)
        if (!(cost[p] > 0.0)) return HB_ERR_ARG;
    std::vector<std::vector<int>> mds(n_mds);
    for (int m = 0; m < n_mds; m++) {
        if (md_start[m + 1] < md_start[m]) return HB_ERR_ARG;
        for (int k = md_start[m]; k < md_start[m + 1]; k++) {
            if (md_pred[k] < 0 || md_pred[k] >= n_preds) return HB_ERR_ARG;
            mds[m].push_back(md_pred[k]);
        }
    }
    std::vector<uint8_t> sk(n_preds, 0);
    if (skip)
        for (int p = 0; p < n_preds; p++) sk[p] = skip[p];
    hb::PlanResult R = hb::make_plan(n_preds, sp, cost, mds, sk);
    if (program_out)
        for (size_t i = 0; i < R.program.size(); i++) program_out[i] = R.program[i];
    if (n_prog_out) *n_prog_out = (int32_t)R.program.size();
    if (cp_out)
        for (int m = 0; m < n_mds; m++) cp_out[m] = R.cp[m];
    if (md_order_out)
        for (size_t i = 0; i < R.md_order.size(); i++) md_order_out[i] = R.md_order[i];
    return HB_OK;
}
