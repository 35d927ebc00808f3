// Host-only driver over the TTM launch planning of ttm_plan.h, for the CPU
// tests of the split-K scratch bound.  Reads commands from stdin, one per line:
//   k ctas_xy tpb K num_sms outn part_elems   -> "<splits> <scratch elems>"
//   s N d_0 .. d_{N-1} R n num_sms capacity  -> "<ok> <s0> <s1> <part> <peak> <max splits>"
//   w R                                      -> "<register width of the row kernels>"
#include <stdio.h>

#include "ttm_plan.h"

int main()
{
    char cmd[8];
    while (scanf("%7s", cmd) == 1) {
        if (cmd[0] == 'k') {
            long long ctas, K, outn, part;
            int tpb, sms;
            if (scanf("%lld %d %lld %d %lld %lld", &ctas, &tpb, &K, &sms, &outn, &part) != 6) return 2;
            const int64_t ks = cpals::ttm_ksplit(ctas, tpb, K, sms, outn, part, true);
            printf("%lld %lld\n", (long long)ks, (long long)cpals::ksplit_scratch_elems(ks, outn));
        } else if (cmd[0] == 's') {
            int N, R, n, sms;
            long long cap;
            int64_t dims[cpals::kMaxN];
            if (scanf("%d", &N) != 1 || N < 1 || N > cpals::kMaxN) return 2;
            for (int m = 0; m < N; ++m) {
                long long d;
                if (scanf("%lld", &d) != 1) return 2;
                dims[m] = d;
            }
            if (scanf("%d %d %d %lld", &R, &n, &sms, &cap) != 4) return 2;
            const cpals::StaticPlan p = cpals::plan_multi_ttm_static(N, dims, R, n, sms, cap);
            printf("%d %lld %lld %lld %lld %lld\n", p.ok ? 1 : 0, (long long)p.s0, (long long)p.s1,
                   (long long)p.part_elems, (long long)p.peak, (long long)p.max_splits);
        } else if (cmd[0] == 'w') {
            int R;
            if (scanf("%d", &R) != 1) return 2;
            printf("%d\n", cpals::ttm_width(R));
        } else {
            return 2;
        }
        fflush(stdout);
    }
    return 0;
}
