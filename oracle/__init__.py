"""CPU oracle (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
arm may import this package.  It wraps the plain C oracle in oracle.c with
ctypes; nothing in it is shared with the CUDA path.
"""
from .oracle_lib import (OracleEnvs, OracleMachine, alu_adc, alu_sbc, base_cycles,  # noqa: F401
                         build, exp_own, nstep_returns, philox4x32_10, policy_logits, policy_mu, policy_prob,
                         policy_sample, preprocess, vtrace, STATE_BYTES)
