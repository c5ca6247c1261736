"""GB300-native (sm_103a) PAM fitting path: Shepard-normalised Gaussian RBF
surrogates fitted per subdomain by an Elastic Net with residual-driven
refinement, evaluated on arbitrary points.

The compute path is the C-ABI library ``libpam`` (hand-written CUDA, built by
``__graft_entry__.build()``); ``paper_2605_16564_gb300.pam`` is its thin
Python binding. ``fields`` draws the seeded synthetic inputs.
"""
