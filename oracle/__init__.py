"""serialWT oracle: test infrastructure only (see serialwt.c)."""
