"""FP64 CPU oracle (test infrastructure only; never imported by the product path).

See lsm_oracle.py for what it computes and which passage of the paper each part follows.
"""
