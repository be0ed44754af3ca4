/* gmg_oracle_amr.c -- two-level composite solve and adjoint for the oracle
   (filled in with the two-level composite form; empty translation unit until then). */
typedef int orc_amr_placeholder_t;
