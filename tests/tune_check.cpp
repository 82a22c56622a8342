// The launch-variant tuning table and selection rule (csrc/st_tune.h) on the
// CPU: round reduction, the margin that keeps the built-in choice, invalid
// variants, and concurrent lookups while entries are added.  Built and run
// by tests/test_tune_table.py; prints one line per check and PASS at the end.
#include <cmath>
#include <cstdio>
#include <thread>
#include <vector>

#include "st_tune.h"

namespace {

int failures = 0;

void check(bool ok, const char* what) {
    std::printf("%s %s\n", ok ? "ok  " : "FAIL", what);
    if (!ok) ++failures;
}

}  // namespace

int main() {
    using namespace sttune;
    // rounds x variants; the first round (cold) is ignored, the best later round kept
    {
        const double t[4 * 3] = {9.0, 9.0, 9.0,   //
                                 2.0, 3.0, -1.0,  //
                                 1.5, 3.5, -1.0,  //
                                 1.8, 2.9, -1.0};
        double ms[3];
        reduce_rounds(t, 4, 3, ms);
        check(ms[0] == 1.5 && ms[1] == 2.9 && ms[2] == -1.0, "reduce_rounds: best of rounds 1.., invalid stays -1");
        const double one[3] = {1.0, 2.0, 3.0};
        reduce_rounds(one, 1, 3, ms);
        check(ms[0] == -1.0 && ms[1] == -1.0 && ms[2] == -1.0, "reduce_rounds: a warm-up round alone measures nothing");
        const double nanr[2 * 2] = {1.0, 1.0, NAN, 2.0};
        reduce_rounds(nanr, 2, 2, ms);
        check(ms[0] == -1.0 && ms[1] == 2.0, "reduce_rounds: a non-finite round invalidates the variant");
    }
    {
        const double ms[3] = {0.98, 1.00, 1.20};
        check(pick(ms, 3, 1, 0.03) == 1, "pick: 2% faster than the built-in choice keeps it");
        const double ms2[3] = {0.90, 1.00, 1.20};
        check(pick(ms2, 3, 1, 0.03) == 0, "pick: 10% faster replaces it");
        const double ms3[3] = {-1.0, 1.00, 0.50};
        check(pick(ms3, 3, 0, 0.03) == 2, "pick: an unmeasured built-in choice loses to the fastest");
        const double ms4[3] = {-1.0, -1.0, -1.0};
        check(pick(ms4, 3, 1, 0.03) == 1, "pick: nothing measured keeps the built-in choice");
        const double ms5[3] = {0.7, 0.7, 1.0};
        check(pick(ms5, 3, 2, 0.03) == 0, "pick: ties go to the lowest index");
    }
    {
        Table t;
        const Key a{FOLD, 8, 0, 255, 255, 2}, b{FOLD, 8, 1, 255, 255, 2}, c{LINE, 4, 255, 510, 2, 0};
        check(t.size() == 0 && t.get(a) == -1, "table: empty");
        t.put(a, 2);
        t.put(c, 0);
        check(t.get(a) == 2 && t.get(b) == -1 && t.get(c) == 0 && t.size() == 2, "table: keys differ in every field");
        t.put(a, 1);
        check(t.get(a) == 1 && t.size() == 2, "table: a key is overwritten, not duplicated");
        t.clear();
        check(t.size() == 0 && t.get(a) == -1 && t.get(c) == -1, "table: clear");
    }
    {
        // readers and writers on several threads: every read is absent or the value written
        Table t;
        std::vector<std::thread> th;
        std::vector<int> bad(8, 0);
        for (int w = 0; w < 8; ++w)
            th.emplace_back([&, w] {
                for (int i = 0; i < 2000; ++i) {
                    const Key k{FOLD, 8, w % 2, i % 97, w, 1};
                    if (w < 4) t.put(k, (i % 97) % 3);
                    const int v = t.get(Key{FOLD, 8, (w + 1) % 2, i % 97, (w + 1) % 8, 1});
                    if (v != -1 && v != (i % 97) % 3) ++bad[w];
                }
            });
        for (auto& x : th) x.join();
        int nbad = 0;
        for (int v : bad) nbad += v;
        check(nbad == 0 && t.size() == 4 * 97, "table: concurrent puts and gets");
    }
    {
        // the process-wide instance is one object
        table().clear();
        table().put(Key{LINE, 8, 63, 100, 3, 0}, 1);
        check(&table() == &table() && table().size() == 1, "table(): one process-wide instance");
        table().clear();
    }
    std::printf("%s\n", failures ? "FAILED" : "PASS");
    return failures ? 1 : 0;
}
