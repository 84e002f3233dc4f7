// Autotuning of the back-transformation's kernel choice and blocking,
// modelled on the paper's autotuning (Sec. 4.3): a tuning object walks a
// fixed list of settings, the caller runs one solve (here: one
// back-transformation) per setting and reports how long it took, and at the
// end the fastest setting is kept.  The walk can be saved to a text file and
// resumed, so that it can be spread over the iterations of an application's
// self-consistency loop (Sec. 5.3).
//   FAST   : the kernel variant only (wavefront, pipeline, tensor-core pipeline)
//   MEDIUM : the variant and its blocking (sweeps per tile, columns per block;
//            column batch for the tensor-core pipeline)
// Host code only; no device memory is touched.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "elpa_gb300.h"

struct gb_autotune {
    int level, n, nbw, nev;
    std::vector<gb_trans_ev_opts> cand;
    std::vector<double> secs;  // < 0: not measured yet
    int next;                  // index of the next candidate to hand out
    int pending;               // candidate handed out and not yet reported (-1: none)
};

namespace {

bool pipeline_ok(int nbw) { return nbw == 8 || nbw == 16 || nbw == 32 || nbw == 64; }
bool tc_ok(int nbw) { return nbw == 16 || nbw == 32 || nbw == 64; }

void build_candidates(gb_autotune *t)
{
    t->cand.clear();
    auto add = [&](int variant, int nb, int cols, int batch = 0) {
        gb_trans_ev_opts o;
        memset(&o, 0, sizeof(o));
        o.variant = variant;
        o.sweeps_per_tile = nb;
        o.cols_per_block = cols;
        o.column_batch = batch;
        t->cand.push_back(o);
    };
    const bool real_reg = t->nbw <= 64;
    if (t->level == GB_AUTOTUNE_FAST) {
        add(GB_VARIANT_WAVEFRONT, 0, 0);
        if (pipeline_ok(t->nbw)) add(GB_VARIANT_PIPELINE, 0, 0);
        if (tc_ok(t->nbw)) add(GB_VARIANT_PIPELINE_TC, 0, 0);
        if (tc_ok(t->nbw)) add(GB_VARIANT_PIPELINE_TC5, 0, 0);
    } else {
        const int wnb[3] = {4, 8, 16}, wcols[3] = {32, 64, 128};
        for (int a = 0; a < 3; a++)
            for (int c = 0; c < 3; c++)
                if (real_reg || wcols[c] <= 64) add(GB_VARIANT_WAVEFRONT, wnb[a], wcols[c]);
        if (pipeline_ok(t->nbw)) {
            const int pnb[2] = {8, 16}, pcols[2] = {64, 128};
            for (int a = 0; a < 2; a++)
                for (int c = 0; c < 2; c++) add(GB_VARIANT_PIPELINE, pnb[a], pcols[c]);
        }
        if (tc_ok(t->nbw)) {
            const int tcb[3] = {8, 16, 32};
            for (int a = 0; a < 3; a++) add(GB_VARIANT_PIPELINE_TC, 0, 0, tcb[a]);
            const int tc5b[3] = {2, 4, 8};  // 128-column blocks per batch
            for (int a = 0; a < 3; a++) add(GB_VARIANT_PIPELINE_TC5, 0, 0, tc5b[a]);
        }
    }
    t->secs.assign(t->cand.size(), -1.0);
}

}  // namespace

extern "C" {

gb_autotune *gb_autotune_create(int level, int n, int nbw, int nev)
{
    if ((level != GB_AUTOTUNE_FAST && level != GB_AUTOTUNE_MEDIUM) || n < 1 || nbw < 1 || nev < 0) return NULL;
    gb_autotune *t = new gb_autotune;
    t->level = level;
    t->n = n;
    t->nbw = nbw;
    t->nev = nev;
    t->next = 0;
    t->pending = -1;
    build_candidates(t);
    return t;
}

void gb_autotune_destroy(gb_autotune *t) { delete t; }

int gb_autotune_step(gb_autotune *t, gb_trans_ev_opts *next)
{
    if (!t) return -1;
    if (!next) return -2;
    if (t->pending >= 0) return -1;  // report the previous candidate first
    if (t->next >= (int)t->cand.size()) return 0;
    *next = t->cand[t->next];
    t->pending = t->next++;
    return 1;
}

int gb_autotune_report(gb_autotune *t, double seconds)
{
    if (!t || t->pending < 0) return -1;
    if (!(seconds >= 0.0)) return -2;
    t->secs[t->pending] = seconds;
    t->pending = -1;
    return 0;
}

int gb_autotune_best(const gb_autotune *t, gb_trans_ev_opts *best, double *seconds)
{
    if (!t) return -1;
    if (!best) return -2;
    int bi = -1;
    for (size_t i = 0; i < t->secs.size(); i++)
        if (t->secs[i] >= 0.0 && (bi < 0 || t->secs[i] < t->secs[bi])) bi = (int)i;
    if (bi < 0) return GB_ERR_UNSUPPORTED;  // nothing measured yet
    *best = t->cand[bi];
    if (seconds) *seconds = t->secs[bi];
    return GB_OK;
}

int gb_autotune_progress(const gb_autotune *t, int *tried, int *total)
{
    if (!t) return -1;
    if (tried) *tried = t->next;
    if (total) *total = (int)t->cand.size();
    return GB_OK;
}

int gb_autotune_save(const gb_autotune *t, const char *path)
{
    if (!t) return -1;
    if (!path) return -2;
    FILE *f = fopen(path, "w");
    if (!f) return GB_ERR_UNSUPPORTED;
    // a candidate handed out but not reported yet is tried again on resume
    const int next = t->pending >= 0 ? t->pending : t->next;
    fprintf(f, "gb_autotune 2\nlevel %d\nn %d\nnbw %d\nnev %d\nnext %d\ncandidates %zu\n", t->level, t->n, t->nbw,
            t->nev, next, t->cand.size());
    for (size_t i = 0; i < t->cand.size(); i++)
        fprintf(f, "c %d %d %d %d %.17g\n", t->cand[i].variant, t->cand[i].sweeps_per_tile, t->cand[i].cols_per_block,
                t->cand[i].column_batch, t->secs[i]);
    int rc = fclose(f);
    return rc == 0 ? GB_OK : GB_ERR_UNSUPPORTED;
}

gb_autotune *gb_autotune_load(const char *path)
{
    if (!path) return NULL;
    FILE *f = fopen(path, "r");
    if (!f) return NULL;
    int ver = 0, level = 0, n = 0, nbw = 0, nev = 0, next = 0;
    size_t ncand = 0;
    gb_autotune *t = NULL;
    if (fscanf(f, "gb_autotune %d level %d n %d nbw %d nev %d next %d candidates %zu", &ver, &level, &n, &nbw, &nev,
               &next, &ncand) == 7 &&
        ver == 2) {
        t = gb_autotune_create(level, n, nbw, nev);
        if (t && ncand == t->cand.size() && next >= 0 && next <= (int)ncand) {
            for (size_t i = 0; i < ncand; i++) {
                int v, nb, cols, cb;
                double s;
                if (fscanf(f, " c %d %d %d %d %lg", &v, &nb, &cols, &cb, &s) != 5 || v != t->cand[i].variant ||
                    nb != t->cand[i].sweeps_per_tile || cols != t->cand[i].cols_per_block ||
                    cb != t->cand[i].column_batch) {
                    delete t;
                    t = NULL;
                    break;
                }
                t->secs[i] = s;
            }
            if (t) t->next = next;
        } else if (t) {
            delete t;
            t = NULL;
        }
    }
    fclose(f);
    return t;
}

}  // extern "C"
