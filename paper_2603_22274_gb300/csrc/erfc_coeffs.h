// Generated by gen_erfc_coeffs.py: erfc(t) ~= u*Q(u)*exp(-t*t), u = 1/(1+0.5 t),
// Q(u) = sum_k ABFE_ERFC_Qk u^k, valid for 0 <= t <= 3.6 (own Chebyshev fit).
#pragma once
#define ABFE_ERFC_PSUB 0.5f
#define ABFE_ERFC_TMAX 3.6
#define ABFE_ERFC_DEG 7
#define ABFE_ERFC_Q0 (2.835482485e-01f)
#define ABFE_ERFC_Q1 (2.625252102e-01f)
#define ABFE_ERFC_Q2 (3.587438714e-01f)
#define ABFE_ERFC_Q3 (-1.748156075e-01f)
#define ABFE_ERFC_Q4 (7.288393972e-01f)
#define ABFE_ERFC_Q5 (-6.713976566e-01f)
#define ABFE_ERFC_Q6 (2.450680095e-01f)
#define ABFE_ERFC_Q7 (-3.251144600e-02f)
